/*
 * hpf_oracle.c -- plain CPU oracle of the hybrid particle-field (MD-SCF) step.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline leg of the benchmark, never by the product path.  Shares no code
 * with the CUDA library.  Written for readability, not speed: every function
 * is a direct transcription of the definition it cites.  Compile with
 * -ffp-contract=off so no multiply-add is fused behind our back.
 *
 * Paper: Zhu et al., "GALAMOST: GPU-accelerated large-scale molecular
 * simulation toolkit", section "The MD-SCF treatment of interparticle forces"
 * (external potential V_K, the two-component V_A and the force F_A = -dV_A/dr),
 * section "Bonded forces" (U_bond = k (r - r0)^2, no factor 1/2), section
 * "Integration methods" (velocity-Verlet), Algorithm 1 kernels 1-4.
 *
 * Readings where the paper is silent (all listed with their reasons in the
 * design notes of the repository):
 *   - phi_K = rho_K / rho0, so the count of species K at a node becomes
 *     phi = count / (rho0 * cell volume); V_K = kT sum_K' chi_KK' phi_K'
 *     + inv_kappa (sum_K phi_K - 1) with chi in kT units.
 *   - CIC vertices sit at integer multiples of h; a bead in cell i feeds
 *     nodes i and i+1 (mod M) per axis (Algorithm 1, kernel 2: "eight
 *     vertices of the cell in which the particle resides").
 *   - The density is accumulated as fixed point: per axis the weight of the
 *     upper node is q = floor(2^13 frac(s)) and of the lower node 2^13 - q,
 *     where s = fl32(fl32(x) * fl32(M / L)) is the mesh coordinate, so one
 *     bead adds exactly 2^39 to the mesh.
 *   - Gradients are central differences at the nodes (the mean of the
 *     backward and forward differences of Algorithm 1, kernel 3), and the
 *     force at a bead is the trilinear interpolation of the nodal gradient of
 *     its own species with the same vertex convention (kernel 4).
 *   - Velocity-Verlet is used in its kick-drift form with the two half kicks
 *     between drifts merged; the state velocity is the half-step velocity
 *     v_{n-1/2}.  A Langevin force -gamma m v + sqrt(2 gamma m kT / dt) xi
 *     is added to the force (the thermostat the paper lists is Nose-Hoover /
 *     Andersen; the Langevin form and its Philox noise are this library's).
 */
#include "hpf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ONE_Q ((int64_t)1 << ORC_FRAC_BITS) /* 8192: fixed-point weight of a whole axis */

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ Philox */

/* Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11): ten rounds of the S-box built from two
 * 32x32->64 multiplications, with a Weyl-sequence key schedule. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform in (0,1): the top 23 bits as an odd multiple of 2^-24. */
static double uniform_open(uint32_t r)
{
    return (double)(2u * (r >> 9) + 1u) * ldexp(1.0, -24);
}

/* Gaussian noise of bead `tag` at step `step`: counter (tag, step lo, step hi, 0),
 * key (seed lo, seed hi); Box-Muller on (u0,u1) gives x and y, on (u2,u3) gives z. */
void orc_gauss3(uint64_t seed, uint32_t tag, int64_t step, double xi[3])
{
    const double two_pi = 6.283185307179586476925286766559;
    uint64_t us = (uint64_t)step;
    uint32_t ctr[4] = {tag, (uint32_t)us, (uint32_t)(us >> 32), 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    double u0 = uniform_open(r[0]), u1 = uniform_open(r[1]);
    double u2 = uniform_open(r[2]), u3 = uniform_open(r[3]);
    double a = sqrt(-2.0 * log(u0));
    double b = sqrt(-2.0 * log(u2));
    xi[0] = a * cos(two_pi * u1);
    xi[1] = a * sin(two_pi * u1);
    xi[2] = b * cos(two_pi * u3);
}

int orc_andersen_collides(const orc_params* p, uint32_t tag, int64_t step)
{
    uint64_t us = (uint64_t)step;
    uint32_t ctr[4] = {tag, (uint32_t)us, (uint32_t)(us >> 32), 1u};
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    const float u = (float)uniform_open(r[0]);
    return u < (float)(p->andersen_nu * p->dt);
}

/* ------------------------------------------------------------ mesh helpers */

float orc_inv_h(const orc_params* p, int axis)
{
    return (float)((double)p->mesh[axis] / (double)p->box[axis]);
}

static int64_t wrap(int64_t i, int64_t m)
{
    int64_t r = i % m;
    return r < 0 ? r + m : r;
}

static int64_t n_nodes(const orc_params* p)
{
    return (int64_t)p->mesh[0] * p->mesh[1] * p->mesh[2];
}

static int64_t node_index(const orc_params* p, int64_t x, int64_t y, int64_t z)
{
    return (z * p->mesh[1] + y) * p->mesh[0] + x;
}

/* Mesh coordinate of one component: lower and upper node, fixed-point weight
 * q of the upper node, and the exact fractional offset f. */
typedef struct {
    int64_t lo, hi, q;
    double f;
} axis_coord;

static axis_coord mesh_coord(const orc_params* p, int axis, double x)
{
    float xf = (float)x;
    float s = xf * orc_inv_h(p, axis); /* one FP32 multiply */
    double sd = (double)s;
    double fl = floor(sd);
    /* q = floor(2^13 frac(s)) evaluated without rounding: 2^13 s is exact, so
     * q = floor(2^13 s) - 2^13 floor(s).  (s - floor(s) itself rounds when s is
     * a tiny negative number, e.g. 1 - 1e-30 -> 1.) */
    double t = floor(sd * (double)ONE_Q);
    axis_coord c;
    c.q = (int64_t)t - (int64_t)fl * ONE_Q;
    c.f = sd - fl; /* interpolation weight */
    c.lo = wrap((int64_t)fl, p->mesh[axis]);
    c.hi = wrap((int64_t)fl + 1, p->mesh[axis]);
    return c;
}

/* ------------------------------------------------------------ A2: density */

/* Cloud-in-cell assignment of each bead to the eight vertices of its cell
 * (MD-SCF section; Algorithm 1, kernels 1-2 compute the same sums by
 * gathering per vertex).  Integer sums, so any order gives the same mesh. */
void orc_scatter(const orc_params* p, int64_t n, const double* pos, const int32_t* type,
                 int64_t* D)
{
    int64_t M = n_nodes(p);
    memset(D, 0, sizeof(int64_t) * (size_t)(M * p->n_species));
    for (int64_t i = 0; i < n; ++i) {
        axis_coord c[3];
        for (int a = 0; a < 3; ++a) c[a] = mesh_coord(p, a, pos[3 * i + a]);
        int64_t wx[2] = {ONE_Q - c[0].q, c[0].q};
        int64_t wy[2] = {ONE_Q - c[1].q, c[1].q};
        int64_t wz[2] = {ONE_Q - c[2].q, c[2].q};
        int64_t nx[2] = {c[0].lo, c[0].hi};
        int64_t ny[2] = {c[1].lo, c[1].hi};
        int64_t nz[2] = {c[2].lo, c[2].hi};
        int64_t* Dk = D + (int64_t)type[i] * M;
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx)
                    Dk[node_index(p, nx[dx], ny[dy], nz[dz])] += wx[dx] * wy[dy] * wz[dz];
    }
}

/* Normalised density phi = count / (rho0 * cell volume); count = D / 2^39. */
static double phi_scale(const orc_params* p)
{
    double vol = 1.0;
    for (int a = 0; a < 3; ++a) vol *= (double)p->box[a] / (double)p->mesh[a];
    return ldexp(1.0, -3 * ORC_FRAC_BITS) / (p->rho0 * vol);
}

/* ------------------------------------------------------------ A3: field */

/* External potential of the MD-SCF section,
 *   V_K = kT sum_K' chi_KK' phi_K' + inv_kappa (sum_K phi_K - 1),
 * then its gradient by central differences (Algorithm 1, kernel 3 stores the
 * backward and forward differences; their mean is the central difference). */
void orc_field(const orc_params* p, const int64_t* D, double* V, double* G)
{
    const int S = p->n_species;
    const int64_t M = n_nodes(p);
    const double c = phi_scale(p);
#pragma omp parallel for schedule(static)
    for (int64_t node = 0; node < M; ++node) {
        double phi[ORC_MAX_SPECIES];
        double total = 0.0;
        for (int k = 0; k < S; ++k) {
            phi[k] = c * (double)D[k * M + node];
            total += phi[k];
        }
        for (int k = 0; k < S; ++k) {
            double v = 0.0;
            for (int kp = 0; kp < S; ++kp) v += p->kT * p->chi[k * ORC_MAX_SPECIES + kp] * phi[kp];
            v += p->inv_kappa * (total - 1.0);
            V[k * M + node] = v;
        }
    }
    double h[3];
    for (int a = 0; a < 3; ++a) h[a] = (double)p->box[a] / (double)p->mesh[a];
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < p->mesh[2]; ++z)
        for (int64_t y = 0; y < p->mesh[1]; ++y)
            for (int64_t x = 0; x < p->mesh[0]; ++x) {
                int64_t node = node_index(p, x, y, z);
                int64_t xp = node_index(p, wrap(x + 1, p->mesh[0]), y, z);
                int64_t xm = node_index(p, wrap(x - 1, p->mesh[0]), y, z);
                int64_t yp = node_index(p, x, wrap(y + 1, p->mesh[1]), z);
                int64_t ym = node_index(p, x, wrap(y - 1, p->mesh[1]), z);
                int64_t zp = node_index(p, x, y, wrap(z + 1, p->mesh[2]));
                int64_t zm = node_index(p, x, y, wrap(z - 1, p->mesh[2]));
                for (int k = 0; k < S; ++k) {
                    const double* Vk = V + k * M;
                    double* g = G + 3 * (k * M + node);
                    g[0] = (Vk[xp] - Vk[xm]) / (2.0 * h[0]);
                    g[1] = (Vk[yp] - Vk[ym]) / (2.0 * h[1]);
                    g[2] = (Vk[zp] - Vk[zm]) / (2.0 * h[2]);
                }
            }
}

/* ------------------------------------------------------------ A4: gather */

/* F = -grad V_T at the bead, trilinear in the nodal gradients of its species T
 * (force equation F_A = -dV_A/dr of the MD-SCF section; Algorithm 1, kernel 4). */
void orc_field_force(const orc_params* p, int64_t n, const double* pos, const int32_t* type,
                     const double* G, double* F)
{
    const int64_t M = n_nodes(p);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        axis_coord c[3];
        for (int a = 0; a < 3; ++a) c[a] = mesh_coord(p, a, pos[3 * i + a]);
        double wx[2] = {1.0 - c[0].f, c[0].f};
        double wy[2] = {1.0 - c[1].f, c[1].f};
        double wz[2] = {1.0 - c[2].f, c[2].f};
        int64_t nx[2] = {c[0].lo, c[0].hi};
        int64_t ny[2] = {c[1].lo, c[1].hi};
        int64_t nz[2] = {c[2].lo, c[2].hi};
        const double* Gk = G + 3 * (int64_t)type[i] * M;
        double f[3] = {0.0, 0.0, 0.0};
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    double w = wx[dx] * wy[dy] * wz[dz];
                    const double* g = Gk + 3 * node_index(p, nx[dx], ny[dy], nz[dz]);
                    for (int a = 0; a < 3; ++a) f[a] -= w * g[a];
                }
        for (int a = 0; a < 3; ++a) F[3 * i + a] = f[a];
    }
}

/* Variant: the exact derivative of the CIC field energy with the potential
 * held fixed, F = -sum_c V_T(c) d w_c / d r, where w_c is the (continuous)
 * cloud-in-cell weight of vertex c.  Not the paper's scheme; used to pin
 * energy conservation of the integrator and the V / W pairing. */
void orc_field_force_exact(const orc_params* p, int64_t n, const double* pos, const int32_t* type,
                           const double* V, double* F)
{
    const int64_t M = n_nodes(p);
    double inv_h[3];
    for (int a = 0; a < 3; ++a) inv_h[a] = (double)p->mesh[a] / (double)p->box[a];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        axis_coord c[3];
        for (int a = 0; a < 3; ++a) c[a] = mesh_coord(p, a, pos[3 * i + a]);
        double w[3][2], dw[3][2];
        int64_t nd[3][2];
        for (int a = 0; a < 3; ++a) {
            w[a][0] = 1.0 - c[a].f;
            w[a][1] = c[a].f;
            dw[a][0] = -inv_h[a];
            dw[a][1] = inv_h[a];
            nd[a][0] = c[a].lo;
            nd[a][1] = c[a].hi;
        }
        const double* Vk = V + (int64_t)type[i] * M;
        double f[3] = {0.0, 0.0, 0.0};
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    double v = Vk[node_index(p, nd[0][dx], nd[1][dy], nd[2][dz])];
                    f[0] -= v * dw[0][dx] * w[1][dy] * w[2][dz];
                    f[1] -= v * w[0][dx] * dw[1][dy] * w[2][dz];
                    f[2] -= v * w[0][dx] * w[1][dy] * dw[2][dz];
                }
        for (int a = 0; a < 3; ++a) F[3 * i + a] = f[a];
    }
}

/* The field force of Algorithm 1, kernels 3-4, read literally (force_mode 2).
 * Kernel 3 keeps, per vertex and axis, the backward and forward differences
 * of the density (here of V, into which kernel 4's chi sum folds), which sit
 * half a mesh spacing below and above the vertex; kernel 4 blends them with
 * "fraction ratios" at the bead's vertex.  Reading: the vertex is the one
 * nearest the bead, c = floor(s + 1/2) per axis (s the FP32 mesh coordinate),
 * and the fractions are the linear interpolation weights between the two
 * half-points, xf1 = 1/2 - d and xf2 = 1/2 + d with d = s - c in [-1/2, 1/2):
 *   F_a = -(1/h_a) [xf1 (V(c) - V(c - e_a)) + xf2 (V(c + e_a) - V(c))],
 * only the vertex's own grid line entering each component.  Parity: pinned
 * (quadratic fields exact, central difference on a vertex, continuity between
 * vertices, the sinusoid closed form). */
void orc_field_force_staggered(const orc_params* p, int64_t n, const double* pos,
                               const int32_t* type, const double* V, double* F)
{
    const int64_t M = n_nodes(p);
    double inv_h[3];
    for (int a = 0; a < 3; ++a) inv_h[a] = (double)p->mesh[a] / (double)p->box[a];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3];
        double d[3];
        for (int a = 0; a < 3; ++a) {
            const float s = (float)pos[3 * i + a] * orc_inv_h(p, a); /* as mesh_coord */
            const double r = floor((double)s + 0.5);
            d[a] = (double)s - r;
            c[a] = wrap((int64_t)r, p->mesh[a]);
        }
        const double* Vk = V + (int64_t)type[i] * M;
        const double vc = Vk[node_index(p, c[0], c[1], c[2])];
        for (int a = 0; a < 3; ++a) {
            int64_t m[3] = {c[0], c[1], c[2]}, q[3] = {c[0], c[1], c[2]};
            m[a] = wrap(c[a] - 1, p->mesh[a]);
            q[a] = wrap(c[a] + 1, p->mesh[a]);
            const double vm = Vk[node_index(p, m[0], m[1], m[2])];
            const double vp = Vk[node_index(p, q[0], q[1], q[2])];
            F[3 * i + a] = -inv_h[a] * ((0.5 - d[a]) * (vc - vm) + (0.5 + d[a]) * (vp - vc));
        }
    }
}

/* ------------------------------------------------------------ A5: bonds */

int orc_bond_table(int64_t n, int64_t n_bonds, const int32_t* pairs, int32_t* BL, int32_t* BN)
{
    for (int64_t i = 0; i < n; ++i) BN[i] = 0;
    for (int64_t b = 0; b < n_bonds; ++b) {
        int64_t i = pairs[2 * b], j = pairs[2 * b + 1];
        if (i < 0 || j < 0 || i >= n || j >= n || i == j) return -1;
        if (BN[i] >= ORC_MAX_BONDS || BN[j] >= ORC_MAX_BONDS) return -1;
        BL[(int64_t)BN[i] * n + i] = (int32_t)j;
        BN[i] += 1;
        BL[(int64_t)BN[j] * n + j] = (int32_t)i;
        BN[j] += 1;
    }
    return 0;
}

/* U = k (r - r0)^2 (section "Bonded forces", no factor 1/2), so the force on
 * bead i from partner j is -2 k (r - r0) (x_i - x_j) / r.  One bead per
 * iteration, each bond seen from both ends, as in the paper's BL/BN scheme. */
void orc_bond_force(const orc_params* p, int64_t n, const double* pos, const int32_t* BL,
                    const int32_t* BN, double* F)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double f[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < BN[i]; ++k) {
            int64_t j = BL[(int64_t)k * n + i];
            double d[3], r2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                d[a] = pos[3 * i + a] - pos[3 * j + a];
                r2 += d[a] * d[a];
            }
            double r = sqrt(r2);
            double s = -2.0 * p->bond_k * (r - p->bond_r0) / r;
            for (int a = 0; a < 3; ++a) f[a] += s * d[a];
        }
        for (int a = 0; a < 3; ++a) F[3 * i + a] = f[a];
    }
}

/* Angles (section "Bonded forces", both forms).  With u = x_a - x_j,
 * w = x_b - x_j and c = u.w / (|u| |w|) = cos theta:
 *   dc/dx_a = w / (|u| |w|) - c u / |u|^2,  dc/dx_b = u / (|u| |w|) - c w / |w|^2,
 *   dc/dx_j = -(dc/dx_a + dc/dx_b).
 * Cosine form, U = k (c - cos0)^2: F = -2k (c - cos0) dc/dx on each bead.
 * Harmonic form, U = k (theta - theta0)^2 with theta = atan2(|u x w|, u.w) in
 * [0, pi]: dtheta/dx = -(1 / sin theta) dc/dx, so F = 2k (theta - theta0) /
 * sin theta dc/dx; at sin theta = 0 the factor is taken as 0 (the straight
 * chain, where dc/dx vanishes too). */
static double angle_cos(const double* pos, int64_t a, int64_t j, int64_t b, double u[3],
                        double w[3], double* uu, double* ww)
{
    double uw = 0.0;
    *uu = 0.0;
    *ww = 0.0;
    for (int d = 0; d < 3; ++d) {
        u[d] = pos[3 * a + d] - pos[3 * j + d];
        w[d] = pos[3 * b + d] - pos[3 * j + d];
        uw += u[d] * w[d];
        *uu += u[d] * u[d];
        *ww += w[d] * w[d];
    }
    return uw / sqrt(*uu * *ww);
}

/* theta = atan2(|u x w|, u.w) of the vectors angle_cos returned. */
static double angle_theta(const double u[3], const double w[3])
{
    const double cx = u[1] * w[2] - u[2] * w[1], cy = u[2] * w[0] - u[0] * w[2],
                 cz = u[0] * w[1] - u[1] * w[0];
    return atan2(sqrt(cx * cx + cy * cy + cz * cz), u[0] * w[0] + u[1] * w[1] + u[2] * w[2]);
}

/* -dU/dc of one angle: the factor of dc/dx in its forces. */
static double angle_factor(const orc_params* p, double c, const double u[3], const double w[3])
{
    if (p->angle_form != 1) return -2.0 * p->angle_k * (c - p->angle_cos0);
    const double th = angle_theta(u, w), s = sin(th);
    return s > 0.0 ? 2.0 * p->angle_k * (th - p->angle_theta0) / s : 0.0;
}

void orc_angle_force(const orc_params* p, int64_t n, const double* pos, const int32_t* BL,
                     const int32_t* BN, double* F)
{
    for (int64_t i = 0; i < 3 * n; ++i) F[i] = 0.0;
    if (p->angle_k == 0.0) return;
    for (int64_t j = 0; j < n; ++j)
        for (int k1 = 0; k1 < BN[j]; ++k1)
            for (int k2 = k1 + 1; k2 < BN[j]; ++k2) {
                const int64_t a = BL[(int64_t)k1 * n + j], b = BL[(int64_t)k2 * n + j];
                double u[3], w[3], uu, ww;
                const double c = angle_cos(pos, a, j, b, u, w, &uu, &ww);
                const double g = angle_factor(p, c, u, w);
                const double inv = 1.0 / sqrt(uu * ww);
                for (int d = 0; d < 3; ++d) {
                    const double da = w[d] * inv - c * u[d] / uu;
                    const double db = u[d] * inv - c * w[d] / ww;
                    F[3 * a + d] += g * da;
                    F[3 * b + d] += g * db;
                    F[3 * j + d] -= g * (da + db);
                }
            }
}

double orc_angle_energy(const orc_params* p, int64_t n, const double* pos, const int32_t* BL,
                        const int32_t* BN)
{
    long double e = 0.0L;
    if (p->angle_k == 0.0) return 0.0;
    for (int64_t j = 0; j < n; ++j)
        for (int k1 = 0; k1 < BN[j]; ++k1)
            for (int k2 = k1 + 1; k2 < BN[j]; ++k2) {
                double u[3], w[3], uu, ww;
                const double c = angle_cos(pos, BL[(int64_t)k1 * n + j], j,
                                           BL[(int64_t)k2 * n + j], u, w, &uu, &ww);
                if (p->angle_form == 1) {
                    const double d = angle_theta(u, w) - p->angle_theta0;
                    e += (long double)(p->angle_k * d * d);
                } else {
                    e += (long double)(p->angle_k * (c - p->angle_cos0) * (c - p->angle_cos0));
                }
            }
    return (double)e;
}

/* The dihedral of the bonded quadruplet (a, j, k, b) and the vectors its
 * force needs (the convention of the header). */
typedef struct {
    double rij[3], rkj[3], rkl[3], m[3], nv[3];
    double phi;
} dihedral_geom;

static void cross3(const double x[3], const double y[3], double z[3])
{
    z[0] = x[1] * y[2] - x[2] * y[1];
    z[1] = x[2] * y[0] - x[0] * y[2];
    z[2] = x[0] * y[1] - x[1] * y[0];
}

static double dot3(const double x[3], const double y[3])
{
    return x[0] * y[0] + x[1] * y[1] + x[2] * y[2];
}

static dihedral_geom dihedral_of(const double* pos, int64_t a, int64_t j, int64_t k, int64_t b)
{
    dihedral_geom q;
    for (int d = 0; d < 3; ++d) {
        q.rij[d] = pos[3 * a + d] - pos[3 * j + d];
        q.rkj[d] = pos[3 * k + d] - pos[3 * j + d];
        q.rkl[d] = pos[3 * k + d] - pos[3 * b + d];
    }
    cross3(q.rij, q.rkj, q.m);
    cross3(q.rkj, q.rkl, q.nv);
    q.phi = atan2(sqrt(dot3(q.rkj, q.rkj)) * dot3(q.rij, q.nv), dot3(q.m, q.nv));
    return q;
}

/* Every bonded quadruplet (a, j, k, b) once: the bond j-k with j < k, a
 * another neighbour of j, b another neighbour of k (b != a).  Returns the
 * count; *out (malloc'd, 4 indices each) holds them. */
static int64_t dihedral_list(int64_t n, const int32_t* BL, const int32_t* BN, int64_t** out)
{
    int64_t cap = 16, cnt = 0;
    int64_t* q = (int64_t*)malloc(sizeof(int64_t) * 4 * (size_t)cap);
    for (int64_t j = 0; j < n; ++j)
        for (int kj = 0; kj < BN[j]; ++kj) {
            const int64_t k = BL[(int64_t)kj * n + j];
            if (k <= j) continue;
            for (int ka = 0; ka < BN[j]; ++ka) {
                const int64_t a = BL[(int64_t)ka * n + j];
                if (a == k) continue;
                for (int kb = 0; kb < BN[k]; ++kb) {
                    const int64_t b = BL[(int64_t)kb * n + k];
                    if (b == j || b == a) continue;
                    if (cnt == cap) {
                        cap *= 2;
                        q = (int64_t*)realloc(q, sizeof(int64_t) * 4 * (size_t)cap);
                    }
                    q[4 * cnt] = a;
                    q[4 * cnt + 1] = j;
                    q[4 * cnt + 2] = k;
                    q[4 * cnt + 3] = b;
                    ++cnt;
                }
            }
        }
    *out = q;
    return cnt;
}

void orc_dihedral_force(const orc_params* p, int64_t n, const double* pos, const int32_t* BL,
                        const int32_t* BN, double* F)
{
    for (int64_t i = 0; i < 3 * n; ++i) F[i] = 0.0;
    if (p->dihedral_k == 0.0) return;
    int64_t* q4 = NULL;
    const int64_t cnt = dihedral_list(n, BL, BN, &q4);
    for (int64_t t = 0; t < cnt; ++t) {
        const int64_t a = q4[4 * t], j = q4[4 * t + 1], k = q4[4 * t + 2], b = q4[4 * t + 3];
        const dihedral_geom q = dihedral_of(pos, a, j, k, b);
        /* dU/dphi */
        const double g = -p->dihedral_k * p->dihedral_n *
                         sin(p->dihedral_n * q.phi - p->dihedral_delta);
        const double rkj2 = dot3(q.rkj, q.rkj), rkj = sqrt(rkj2);
        const double mm = dot3(q.m, q.m), nn = dot3(q.nv, q.nv);
        const double pa = dot3(q.rij, q.rkj) / rkj2, pb = dot3(q.rkl, q.rkj) / rkj2;
        for (int d = 0; d < 3; ++d) {
            const double fa = -g * rkj / mm * q.m[d];
            const double fb = g * rkj / nn * q.nv[d];
            F[3 * a + d] += fa;
            F[3 * b + d] += fb;
            F[3 * j + d] += -fa + pa * fa - pb * fb;
            F[3 * k + d] += -fb - pa * fa + pb * fb;
        }
    }
    free(q4);
}

double orc_dihedral_energy(const orc_params* p, int64_t n, const double* pos, const int32_t* BL,
                           const int32_t* BN)
{
    if (p->dihedral_k == 0.0) return 0.0;
    int64_t* q4 = NULL;
    const int64_t cnt = dihedral_list(n, BL, BN, &q4);
    long double e = 0.0L;
    for (int64_t t = 0; t < cnt; ++t) {
        const dihedral_geom q = dihedral_of(pos, q4[4 * t], q4[4 * t + 1], q4[4 * t + 2],
                                            q4[4 * t + 3]);
        e += (long double)(p->dihedral_k * (1.0 + cos(p->dihedral_n * q.phi - p->dihedral_delta)));
    }
    free(q4);
    return (double)e;
}

double orc_bond_energy(const orc_params* p, int64_t n, const double* pos, const int32_t* BL,
                       const int32_t* BN)
{
    long double e = 0.0L;
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < BN[i]; ++k) {
            int64_t j = BL[(int64_t)k * n + i];
            if (j <= i) continue; /* each bond once */
            double r2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                double d = pos[3 * i + a] - pos[3 * j + a];
                r2 += d * d;
            }
            double dr = sqrt(r2) - p->bond_r0;
            e += (long double)(p->bond_k * dr * dr);
        }
    return (double)e;
}

/* ------------------------------------------------------------ A7: energies */

/* Field energy whose derivative with respect to the bead count of species K
 * at a node is V_K there:
 *   W = rho0 Vc sum_nodes [ 1/2 kT sum_KK' chi_KK' phi_K phi_K'
 *                           + 1/2 inv_kappa (sum_K phi_K - 1)^2 ]. */
double orc_field_energy(const orc_params* p, const int64_t* D)
{
    const int S = p->n_species;
    const int64_t M = n_nodes(p);
    const double c = phi_scale(p);
    double vol = 1.0;
    for (int a = 0; a < 3; ++a) vol *= (double)p->box[a] / (double)p->mesh[a];
    long double w = 0.0L;
    for (int64_t node = 0; node < M; ++node) {
        double phi[ORC_MAX_SPECIES], total = 0.0, e = 0.0;
        for (int k = 0; k < S; ++k) {
            phi[k] = c * (double)D[k * M + node];
            total += phi[k];
        }
        for (int k = 0; k < S; ++k)
            for (int kp = 0; kp < S; ++kp)
                e += 0.5 * p->kT * p->chi[k * ORC_MAX_SPECIES + kp] * phi[k] * phi[kp];
        e += 0.5 * p->inv_kappa * (total - 1.0) * (total - 1.0);
        w += (long double)e;
    }
    return (double)(w * (long double)(p->rho0 * vol));
}

/* Langevin friction coefficient gamma m and noise amplitude; both zero for
 * the other thermostats (Andersen acts on the velocity instead). */
static double friction(const orc_params* p)
{
    return p->thermostat == 0 ? p->gamma * p->mass : 0.0;
}

static double noise_sigma(const orc_params* p)
{
    return p->thermostat == 0 ? sqrt(2.0 * p->gamma * p->mass * p->kT / p->dt) : 0.0;
}

/* Andersen (thermostat 2): the on-step velocity v_n = v + dt/(2m) F_n of a
 * bead that collides at step n is replaced by sqrt(kT/m) xi, xi the three
 * normals of orc_gauss3 at (tag, n).  Returns 1 and writes u[3] if it does. */
static int andersen_velocity(const orc_params* p, int64_t i, int64_t step, double u[3])
{
    if (p->thermostat != 2 || !orc_andersen_collides(p, (uint32_t)i, step)) return 0;
    double xi[3];
    orc_gauss3(p->seed, (uint32_t)i, step, xi);
    const double sv = sqrt(p->kT / p->mass);
    for (int a = 0; a < 3; ++a) u[a] = sv * xi[a];
    return 1;
}

/* Total force at step n on the state (x_n, v_{n-1/2}): conservative part plus
 * Langevin friction on the half-step velocity and Philox noise. */
static void total_force(const orc_params* p, int64_t n, const double* vel, const double* Fc,
                        int64_t step, double* F)
{
    const double sigma = noise_sigma(p);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double xi[3] = {0.0, 0.0, 0.0};
        if (sigma > 0.0) orc_gauss3(p->seed, (uint32_t)i, step, xi);
        for (int a = 0; a < 3; ++a)
            F[3 * i + a] = Fc[3 * i + a] - friction(p) * vel[3 * i + a] + sigma * xi[a];
    }
}

static void conservative_force(const orc_params* p, int64_t n, const double* pos,
                               const int32_t* type, const int32_t* BL, const int32_t* BN,
                               const double* V, const double* G, double* Ff, double* Fb,
                               double* Fc)
{
    if (p->force_mode == 1)
        orc_field_force_exact(p, n, pos, type, V, Ff);
    else if (p->force_mode == 2)
        orc_field_force_staggered(p, n, pos, type, V, Ff);
    else
        orc_field_force(p, n, pos, type, G, Ff);
    orc_bond_force(p, n, pos, BL, BN, Fb);
    if (p->angle_k != 0.0 || p->dihedral_k != 0.0) {
        double* Fa = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
        if (p->angle_k != 0.0) {
            orc_angle_force(p, n, pos, BL, BN, Fa);
            for (int64_t i = 0; i < 3 * n; ++i) Fb[i] += Fa[i];
        }
        if (p->dihedral_k != 0.0) {
            orc_dihedral_force(p, n, pos, BL, BN, Fa);
            for (int64_t i = 0; i < 3 * n; ++i) Fb[i] += Fa[i];
        }
        free(Fa);
    }
    for (int64_t i = 0; i < 3 * n; ++i) Fc[i] = Ff[i] + Fb[i];
}

void orc_energy(const orc_params* p, int64_t n, const double* pos, const double* vel,
                const int32_t* type, const int32_t* BL, const int32_t* BN, const double* V,
                const double* G, int64_t step, double out[6])
{
    double* Ff = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double* Fb = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double* Fc = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double* F = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    int64_t* D = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_nodes(p) * p->n_species));
    conservative_force(p, n, pos, type, BL, BN, V, G, Ff, Fb, Fc);
    total_force(p, n, vel, Fc, step, F);
    /* On-step velocity v_n = v_{n-1/2} + dt/(2m) F_n (mean of the two half steps). */
    long double ke = 0.0L, mom[3] = {0.0L, 0.0L, 0.0L};
    for (int64_t i = 0; i < n; ++i) {
        double u[3];
        const int coll = andersen_velocity(p, i, step, u);
        for (int a = 0; a < 3; ++a) {
            double v = coll ? u[a] : vel[3 * i + a] + 0.5 * p->dt / p->mass * F[3 * i + a];
            ke += (long double)(0.5 * p->mass * v * v);
            mom[a] += (long double)(p->mass * v);
        }
    }
    orc_scatter(p, n, pos, type, D);
    double w = orc_field_energy(p, D);
    /* the bonded entry: bonds, angles and dihedrals */
    double ub = orc_bond_energy(p, n, pos, BL, BN) + orc_angle_energy(p, n, pos, BL, BN) +
                orc_dihedral_energy(p, n, pos, BL, BN);
    out[0] = (double)ke;
    out[1] = ub;
    out[2] = w;
    out[3] = (double)ke + ub + w;
    out[4] = sqrt((double)(mom[0] * mom[0] + mom[1] * mom[1] + mom[2] * mom[2]));
    out[5] = n > 0 ? 2.0 * (double)ke / (3.0 * (double)n) : 0.0;
    free(Ff); free(Fb); free(Fc); free(F); free(D);
}

/* ------------------------------------------------------------ A6: the step */

/* One call advances n_steps steps.  The density field is refreshed from the
 * current positions at the first step of the call and then whenever the step
 * number is a multiple of field_every; in between it is held fixed and only
 * sampled at the moving positions (the quasi-instantaneous field of the
 * MD-SCF section).  Each step, with v the half-step velocity:
 *   F = F_field(x) + F_bond(x) - gamma m v + sqrt(2 gamma m kT / dt) xi(tag, n)
 *   v <- v + dt F / m
 *   x <- x + dt v
 * With the Andersen thermostat (thermostat 2) there is no friction or noise
 * force; a bead that collides at step n (orc_andersen_collides) takes
 *   v <- sqrt(kT/m) xi(tag, n) + dt/(2m) F
 * instead (its on-step velocity redrawn from the Maxwell distribution).
 * Nose-Hoover (thermostat 1) runs through orc_run_nh.                     */
int orc_run(const orc_params* p, int64_t n, double* pos, double* vel, const int32_t* type,
            int64_t n_bonds, const int32_t* pairs, int64_t step0, int32_t n_steps,
            double* energies)
{
    if (p->field_every < 1 || p->n_species < 1 || p->n_species > ORC_MAX_SPECIES || n < 0 ||
        p->force_mode < 0 || p->force_mode > 2 || p->thermostat == 1 ||
        (p->thermostat == 2 && !(p->andersen_nu >= 0.0)))
        return -1;
    size_t nn = (size_t)(n > 0 ? n : 1);
    const int64_t M = n_nodes(p);
    int32_t* BL = (int32_t*)malloc(sizeof(int32_t) * ORC_MAX_BONDS * nn);
    int32_t* BN = (int32_t*)malloc(sizeof(int32_t) * nn);
    if (orc_bond_table(n, n_bonds, pairs, BL, BN) != 0) {
        free(BL); free(BN);
        return -1;
    }
    int64_t* D = (int64_t*)malloc(sizeof(int64_t) * (size_t)(M * p->n_species));
    double* V = (double*)malloc(sizeof(double) * (size_t)(M * p->n_species));
    double* G = (double*)malloc(sizeof(double) * 3 * (size_t)(M * p->n_species));
    double* Ff = (double*)malloc(sizeof(double) * 3 * nn);
    double* Fb = (double*)malloc(sizeof(double) * 3 * nn);
    double* Fc = (double*)malloc(sizeof(double) * 3 * nn);
    double* F = (double*)malloc(sizeof(double) * 3 * nn);
    for (int32_t k = 0; k <= n_steps; ++k) {
        int64_t step = step0 + k;
        if (k == 0 || step % p->field_every == 0) {
            orc_scatter(p, n, pos, type, D);
            orc_field(p, D, V, G);
        }
        if (energies) orc_energy(p, n, pos, vel, type, BL, BN, V, G, step, energies + 6 * k);
        if (k == n_steps) break;
        conservative_force(p, n, pos, type, BL, BN, V, G, Ff, Fb, Fc);
        total_force(p, n, vel, Fc, step, F);
        for (int64_t i = 0; i < n; ++i) {
            double u[3];
            const int coll = andersen_velocity(p, i, step, u);
            for (int a = 0; a < 3; ++a) {
                const int64_t k = 3 * i + a;
                if (coll) vel[k] = u[a] + 0.5 * p->dt * F[k] / p->mass;
                else vel[k] += p->dt * F[k] / p->mass;
                pos[k] += p->dt * vel[k];
            }
        }
    }
    free(BL); free(BN); free(D); free(V); free(G); free(Ff); free(Fb); free(Fc); free(F);
    return 0;
}

/* ------------------------------------------------------------ Nose-Hoover NVT */

static double nh_dof(int64_t n)
{
    return n > 1 ? 3.0 * (double)(n - 1) : 3.0 * (double)n;
}

static double nh_g(const orc_params* p, double dof, double K)
{
    if (dof <= 0.0) return 0.0;
    return (2.0 * K / (dof * p->kT) - 1.0) / (p->nh_tau * p->nh_tau);
}

/* One thermostat half step T(h) of the scheme above; returns the velocity
 * scale and updates xi, eta and the kinetic energy K. */
static double nh_half(const orc_params* p, double dof, double h, double* xi, double* eta,
                      double* K)
{
    *xi += 0.5 * h * nh_g(p, dof, *K);
    const double s = exp(-*xi * h);
    *K *= s * s;
    *eta += *xi * h;
    *xi += 0.5 * h * nh_g(p, dof, *K);
    return s;
}

int orc_run_nh(const orc_params* p, int64_t n, double* pos, double* vel, const int32_t* type,
               int64_t n_bonds, const int32_t* pairs, int64_t step0, int32_t n_steps,
               double xe[2], double* energies)
{
    if (p->field_every < 1 || p->n_species < 1 || p->n_species > ORC_MAX_SPECIES || n < 0 ||
        p->force_mode < 0 || p->force_mode > 2 || !(p->nh_tau > 0.0) || !xe)
        return -1;
    size_t nn = (size_t)(n > 0 ? n : 1);
    const int64_t M = n_nodes(p);
    int32_t* BL = (int32_t*)malloc(sizeof(int32_t) * ORC_MAX_BONDS * nn);
    int32_t* BN = (int32_t*)malloc(sizeof(int32_t) * nn);
    if (orc_bond_table(n, n_bonds, pairs, BL, BN) != 0) {
        free(BL); free(BN);
        return -1;
    }
    int64_t* D = (int64_t*)malloc(sizeof(int64_t) * (size_t)(M * p->n_species));
    double* V = (double*)malloc(sizeof(double) * (size_t)(M * p->n_species));
    double* G = (double*)malloc(sizeof(double) * 3 * (size_t)(M * p->n_species));
    double* Ff = (double*)malloc(sizeof(double) * 3 * nn);
    double* Fb = (double*)malloc(sizeof(double) * 3 * nn);
    double* Fc = (double*)malloc(sizeof(double) * 3 * nn);
    double* vE = (double*)malloc(sizeof(double) * 3 * nn);
    const double dof = nh_dof(n), h = 0.5 * p->dt, hm = 0.5 * p->dt / p->mass;
    double xi = xe[0], eta = xe[1];
    for (int32_t k = 0; k <= n_steps; ++k) {
        int64_t step = step0 + k;
        if (k == 0 || step % p->field_every == 0) {
            orc_scatter(p, n, pos, type, D);
            orc_field(p, D, V, G);
        }
        conservative_force(p, n, pos, type, BL, BN, V, G, Ff, Fb, Fc);
        long double ke = 0.0L;
        for (int64_t i = 0; i < 3 * n; ++i) {
            vE[i] = vel[i] + hm * Fc[i];
            ke += (long double)(0.5 * p->mass * vE[i] * vE[i]);
        }
        double K = (double)ke;
        /* the end of step n - 1 (on copies: the last record's half step is not
           part of the state, which keeps xi, eta at the middle of a step) */
        double xi1 = xi, eta1 = eta;
        const double s1 = nh_half(p, dof, h, &xi1, &eta1, &K);
        if (energies) {
            double* e = energies + 7 * (size_t)k;
            long double mom[3] = {0.0L, 0.0L, 0.0L};
            for (int64_t i = 0; i < n; ++i)
                for (int a = 0; a < 3; ++a) mom[a] += (long double)(p->mass * s1 * vE[3 * i + a]);
            orc_scatter(p, n, pos, type, D);
            const double w = orc_field_energy(p, D);
            const double ub = orc_bond_energy(p, n, pos, BL, BN) +
                              orc_angle_energy(p, n, pos, BL, BN) +
                              orc_dihedral_energy(p, n, pos, BL, BN);
            e[0] = K;
            e[1] = ub;
            e[2] = w;
            e[3] = K + ub + w;
            e[4] = sqrt((double)(mom[0] * mom[0] + mom[1] * mom[1] + mom[2] * mom[2]));
            e[5] = n > 0 ? 2.0 * K / (3.0 * (double)n) : 0.0;
            e[6] = e[3] + dof * p->kT * (0.5 * p->nh_tau * p->nh_tau * xi1 * xi1 + eta1);
        }
        if (k == n_steps) break;
        xi = xi1;
        eta = eta1;
        /* the start of step n */
        const double s2 = nh_half(p, dof, h, &xi, &eta, &K);
        for (int64_t i = 0; i < 3 * n; ++i) {
            vel[i] = s2 * (s1 * vE[i]) + hm * Fc[i];
            pos[i] += p->dt * vel[i];
        }
    }
    xe[0] = xi;
    xe[1] = eta;
    free(BL); free(BN); free(D); free(V); free(G); free(Ff); free(Fb); free(Fc); free(vE);
    return 0;
}

/* ------------------------------------------------------------ A1: order */

/* Sort key of a chain: the cell of its first bead, numbered brick by brick
 * (bricks of `brick`^3 cells, x fastest within and across bricks). */
int64_t orc_cell_key(const orc_params* p, const double* x, int32_t brick)
{
    int64_t cell[3], nb[3];
    for (int a = 0; a < 3; ++a) {
        axis_coord c = mesh_coord(p, a, x[a]);
        cell[a] = c.lo;
        nb[a] = (p->mesh[a] + brick - 1) / brick;
    }
    int64_t b = ((cell[2] / brick) * nb[1] + cell[1] / brick) * nb[0] + cell[0] / brick;
    int64_t in = ((cell[2] % brick) * brick + cell[1] % brick) * brick + cell[0] % brick;
    return b * (int64_t)brick * brick * brick + in;
}
