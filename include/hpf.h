/*
 * hpf.h -- C ABI of the GB300 hybrid particle-field MD (hPF-MD / MD-SCF) library.
 *
 * One context simulates one periodic box of bead-spring polymers whose
 * non-bonded interactions go through a density field, as in the MD-SCF
 * section of Zhu et al., "GALAMOST: GPU-accelerated large-scale molecular
 * simulation toolkit" (the external potential V_K, the force F_A = -dV_A/dr,
 * Algorithm 1), with harmonic bonds (section "Bonded forces") and
 * velocity-Verlet integration (section "Integration methods") plus a
 * Langevin thermostat driven by Philox4x32-10 noise.
 *
 * Conventions that hold for every call:
 *   - All arithmetic runs on the GPU, in kernels enqueued on the CUDA stream
 *     given to hpf_init.  Calls return without waiting for the GPU unless a
 *     call says it synchronises.
 *   - Array arguments are plain pointers that may point to host memory
 *     (pageable or pinned) or to device memory of the context's GPU; the
 *     library copies through them with cudaMemcpyDefault.  The caller keeps
 *     ownership; the library never retains a caller pointer after a call.
 *   - Bead arrays are indexed by the bead tag 0 .. n_beads-1 (the caller's
 *     order).  The library reorders beads internally; every output is
 *     returned in tag order and no result depends on the internal order.
 *   - Layouts are C order: positions, velocities, forces [n_beads][3] float32;
 *     density [n_species][Mz][My][Mx] int64; field [n_species][Mz][My][Mx][4]
 *     float32 = (dV/dx, dV/dy, dV/dz, V).
 *   - Every call returns an hpf_status.  Nothing aborts the process.  The text
 *     of the last failure of a context is kept until the next failure and is
 *     returned by hpf_last_error.
 */
#ifndef HPF_H
#define HPF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HPF_MAX_SPECIES 8
#define HPF_FRAC_BITS 13              /* fixed-point bits of a CIC weight per axis */
#define HPF_MAX_BEADS ((1 << 24) - 1) /* keeps the whole-mesh sum below 2^63 */

typedef enum {
    HPF_OK = 0,
    HPF_ERR_INVALID = 1,   /* bad argument or parameter; nothing was changed */
    HPF_ERR_CUDA = 2,      /* a CUDA runtime call failed; see hpf_last_error */
    HPF_ERR_NOMEM = 3,     /* device allocation failed */
    HPF_ERR_OVERFLOW = 4,  /* n_beads >= 2^24, or a bead left the +-2^18-cell range */
    HPF_ERR_NONFINITE = 5, /* a position or velocity became NaN or infinite */
    HPF_ERR_TIMEOUT = 6,   /* a bounded device-side wait gave up */
    HPF_ERR_STATE = 7,     /* the call needs a state (hpf_set_state) first */
    HPF_ERR_SCRATCH = 8    /* the mesh does not fit hpf_field_forces_noalloc's static scratch */
} hpf_status;

typedef struct hpf_ctx hpf_ctx;

/* Physical and numerical parameters of one system. */
typedef struct {
    int32_t n_beads;      /* 0 .. HPF_MAX_BEADS */
    int32_t n_species;    /* 1 .. HPF_MAX_SPECIES */
    int32_t mesh[3];      /* density mesh Mx, My, Mz (>= 2 each) */
    float box[3];         /* periodic box Lx, Ly, Lz; the mesh coordinate of x is
                             fl32(x * fl32(M / L)) */
    double kT;            /* thermal energy */
    double rho0;          /* reference number density: phi_K = rho_K / rho0 */
    double inv_kappa;     /* compressibility term 1/kappa of V_K (energy units) */
    double chi[HPF_MAX_SPECIES * HPF_MAX_SPECIES]; /* chi_KK' in kT units, row K */
    double bond_k;        /* U_bond = bond_k (r - bond_r0)^2 (no factor 1/2) */
    double bond_r0;
    double mass;          /* bead mass m */
    double dt;            /* time step */
    double gamma;         /* Langevin friction; 0 gives plain velocity-Verlet (NVE) */
    uint64_t seed;        /* Philox key of the thermostat noise */
    int32_t field_every;  /* refresh the density field when step % field_every == 0 */
    int32_t sort_every;   /* re-sort beads every this many steps (0: only in hpf_set_state) */
    int32_t force_mode;   /* field force: 0 = the trilinear interpolation of the nodal
                             central-difference gradient (Algorithm 1, kernels 3-4);
                             1 = the exact derivative of the CIC field energy (the gradient
                             of the trilinear interpolant of V; conserves energy);
                             2 = Algorithm 1, kernels 3-4 read literally: per axis the
                             backward and forward differences of V at the vertex c nearest
                             the bead blended by (1/2 - d, 1/2 + d), d = s - c in [-1/2, 1/2)
                             (s the mesh coordinate), only c's grid line entering */
    double angle_k;       /* angle potential U = angle_k (cos theta - angle_cos0)^2 for every */
    double angle_cos0;    /* bonded triplet (section "Bonded forces", cosine form), theta the
                             angle at the middle bead (pi for a straight chain); 0: none */
    int32_t thermostat;   /* 0: Langevin (gamma, seed); 1: Nose-Hoover NVT (nh_tau; gamma and
                             seed unused), see hpf_get_thermostat; 2: Andersen NVT
                             (andersen_nu, seed; gamma unused), see hpf_step */
    double nh_tau;        /* Nose-Hoover relaxation time tau (> 0 when thermostat == 1) */
    double andersen_nu;   /* Andersen collision frequency nu (>= 0 when thermostat == 2) */
    double dihedral_k;    /* dihedral potential U = dihedral_k [1 + cos(n phi - dihedral_delta)]
                             for every run of three consecutive bonds i-j, j-k, k-l along a
                             chain (section "Bonded forces"); phi the angle between the planes
                             (i, j, k) and (j, k, l), signed by the right-hand rule about j -> k,
                             pi for trans and 0 for cis; 0: none */
    int32_t dihedral_n;   /* multiplicity n, 1 .. 6 (checked only when dihedral_k != 0) */
    double dihedral_delta; /* phase delta in radians */
    int32_t angle_form;   /* 0: the cosine form above; 1: the harmonic form of the same
                             section, U = angle_k (theta - angle_theta0)^2, theta in radians
                             from atan2(|u x w|, u.w) (angle_cos0 unused) */
    double angle_theta0;  /* equilibrium angle of the harmonic form, 0 .. pi */
} hpf_params;

/* Text for a status code (static storage). */
const char* hpf_status_string(hpf_status s);

/* Create a context: validate the parameters and allocate the device buffers
 * (state, density mesh, field mesh, sort scratch).  `stream` is a
 * cudaStream_t (NULL for the legacy default stream); all later work of the
 * context is enqueued on it.  On failure *out is NULL.
 * Errors: HPF_ERR_INVALID (bad parameter, out == NULL), HPF_ERR_OVERFLOW
 * (n_beads > HPF_MAX_BEADS), HPF_ERR_NOMEM, HPF_ERR_CUDA. */
hpf_status hpf_init(const hpf_params* params, void* stream, hpf_ctx** out);

/* Free a context and its device buffers (waits for its stream first). NULL is a no-op. */
hpf_status hpf_destroy(hpf_ctx* ctx);

/* Message of the context's last failure ("" if none).  Valid until the next call. */
const char* hpf_last_error(const hpf_ctx* ctx);

/* Load the bead state at step `step` and sort it for locality.
 *   pos   [n][3] unwrapped positions x_n (the box is applied in mesh space)
 *   vel   [n][3] half-step velocities v_{n-1/2} (see hpf_step)
 *   type  [n]    species 0 .. n_species-1
 *   bonds [n_bonds][2] bonded bead pairs.  The library stores chains
 *         contiguously, so every bond must join consecutive tags (i, i+1) and
 *         appear once (section "Bonded forces" stores partners per bead; this
 *         library keeps only linear chains in tag order).
 * Invalidates the density field: the next call that needs it recomputes it
 * from these positions.  Synchronises the stream (validation result).
 * Errors: HPF_ERR_INVALID (NULL array with n > 0, type out of range, bond not
 * (i, i+1), duplicate bond, step < 0), HPF_ERR_NONFINITE, HPF_ERR_CUDA. */
hpf_status hpf_set_state(hpf_ctx* ctx, const float* pos, const float* vel, const int32_t* type,
                         const int32_t* bonds, int64_t n_bonds, int64_t step);

/* Replace positions and velocities ([n][3] float32 in tag order, host or
 * device) and set the step, keeping the species, the bonds and the bead order
 * of the last sort: the light way to continue from modified coordinates
 * (hpf_set_state reloads the topology and re-sorts).  The field of the old
 * positions is dropped; the density of the new ones is deposited in the same
 * pass that puts them into the library's bead order.  Asynchronous: a non-finite value
 * is reported by the next synchronising call (HPF_ERR_NONFINITE), and the
 * caller's buffers must stay unchanged until the stream reaches the call.
 * Errors: HPF_ERR_INVALID, HPF_ERR_STATE (no hpf_set_state yet), HPF_ERR_CUDA. */
hpf_status hpf_update_state(hpf_ctx* ctx, const float* pos, const float* vel, int64_t step);

/* Copy the state out in tag order (either pointer may be NULL) and the step
 * number.  Synchronises the stream.
 * Errors: HPF_ERR_STATE, HPF_ERR_NONFINITE (state became non-finite), HPF_ERR_CUDA. */
/* Pipelined replacement of positions and velocities, for callers that feed
 * a new state every few steps and want its upload to overlap the GPU work of
 * the previous one (double buffering).  hpf_upload_state starts the copy of
 * pos and vel (tag order, [n][3] FP32, host or device; for an overlapped copy
 * from the host, pinned memory) into one of two context-owned staging slots
 * on the context's own copy stream and returns at once.  The caller keeps
 * both arrays valid and unchanged until the copy has run, which is certain
 * once hpf_energy or hpf_get_state, called after hpf_apply_state, has
 * returned, or hpf_energy_finish of an hpf_energy_start called after it.
 * The copy is ordered after no other work (it runs on a non-blocking stream
 * so that it can overlap the context's): device-resident inputs must be
 * complete when hpf_upload_state is called (their producer's stream
 * synchronised).  hpf_apply_state makes the context's stream wait for that copy and then
 * replaces the state as hpf_update_state(pos, vel, step) does; a slot is
 * reused only after the permutation that read it has run.  One upload may be
 * pending at a time.  Errors: HPF_ERR_INVALID (NULL arrays with n > 0,
 * step < 0), HPF_ERR_STATE (no state; an upload already pending for
 * hpf_upload_state, none for hpf_apply_state), HPF_ERR_CUDA. */
hpf_status hpf_upload_state(hpf_ctx* ctx, const float* pos, const float* vel);
hpf_status hpf_apply_state(hpf_ctx* ctx, int64_t step);

hpf_status hpf_get_state(hpf_ctx* ctx, float* pos, float* vel, int64_t* step);

/* The library's storage order: order[i] is the tag of storage slot i.
 * Whole chains (runs of bonded beads) are kept contiguous and ordered by the
 * cell of their first bead, numbered brick by brick (bricks of 8^3 cells, x
 * fastest inside and across bricks), ties by the first bead's tag.  The
 * order changes at hpf_set_state and every sort_every steps; no result
 * depends on it (the paper sorts particle data for cache locality, section
 * "DPD liquid and LJ liquid").  Synchronises if `order` is host memory.
 * Errors: HPF_ERR_INVALID (order NULL with n > 0), HPF_ERR_STATE, HPF_ERR_CUDA. */
hpf_status hpf_get_order(hpf_ctx* ctx, int32_t* order);

/* Cloud-in-cell density of the current positions (MD-SCF section; Algorithm 1,
 * kernels 1-2): every bead adds w_x w_y w_z to the eight vertices of its cell,
 * with per-axis fixed-point weights (2^13 - q, q), q = floor(2^13 frac(s)),
 * s the mesh coordinate; one bead adds exactly 2^39.  Integer sums make the
 * mesh independent of summation order.  The result stays in the context's
 * mesh and is copied to D_out [n_species][Mz][My][Mx] int64 if D_out != NULL.
 * Errors: HPF_ERR_STATE, HPF_ERR_CUDA. */
hpf_status hpf_scatter_density(hpf_ctx* ctx, int64_t* D_out);

/* Field of a density mesh (MD-SCF section, V_K equation; Algorithm 1, kernel 3):
 *   phi_K = D_K 2^-39 / (rho0 h_x h_y h_z),
 *   V_K   = kT sum_K' chi_KK' phi_K' + inv_kappa (sum_K phi_K - 1),
 *   grad V_K by periodic central differences at the nodes.
 * Uses D_in [n_species][Mz][My][Mx] if not NULL, else the context's mesh (the
 * last hpf_scatter_density or field refresh).  The field becomes the frozen
 * field of the current step; it is copied to field_out if not NULL.
 * Errors: HPF_ERR_STATE, HPF_ERR_CUDA. */
hpf_status hpf_field(hpf_ctx* ctx, const int64_t* D_in, float* field_out);

/* Self-test of the device-side wait bound: one kernel waits on a barrier that
 * nothing completes, which must give up after its limit (0.2 s), raise the
 * context's timeout flag and return.  The flag is cleared again, so the
 * context stays usable; *seconds (may be NULL) is the host-measured time.
 * Returns HPF_ERR_TIMEOUT when the wait gave up as designed, HPF_OK if it
 * completed (the bound did not act).  Synchronises.
 * Errors: HPF_ERR_INVALID, HPF_ERR_CUDA. */
hpf_status hpf_selftest_timeout(hpf_ctx* ctx, double* seconds);

/* The field stencil runs on shared-memory tiles of the mesh, staged by TMA
 * tensor copies when the mesh allows it (Mx even, n_species <= 4), or untiled
 * (one ghosted node, or two real nodes, per thread).  The kernel is chosen
 * the first time the field is computed, by timing the eight candidates on
 * this mesh (that first refresh synchronises once).  shape[0..2] = tile
 * (x, y, z); (0, 0, 0) for the one-node untiled kernel (and before the first
 * refresh), (2, 1, 1) for the node-pair kernel; *uses_tma = 1 if the tiles
 * are staged by TMA, 0 otherwise.  Either pointer may be NULL.
 * Errors: HPF_ERR_INVALID. */
hpf_status hpf_field_tile(const hpf_ctx* ctx, int32_t shape[3], int32_t* uses_tma);

/* Pin the stencil to candidate `tile` (0 .. 7: tiles (32,8,4), (32,8,8),
 * (16,16,4), (64,4,4), (16,16,8), (32,4,8), untiled one node per thread,
 * untiled node pairs) instead of autotuning; -1 autotunes again at the next
 * field.  Every candidate computes the same bits.  Errors: HPF_ERR_INVALID. */
hpf_status hpf_set_field_tile(hpf_ctx* ctx, int32_t tile);

#define HPF_FORCE_FIELD 1
#define HPF_FORCE_BOND 2

/* Conservative force on every bead at the current positions, in tag order:
 * F_out [n][3] = (which & HPF_FORCE_FIELD ? -trilinear(grad V_T) : 0)
 *              + (which & HPF_FORCE_BOND ? -2 k (r - r0) r_hat summed over bonds : 0).
 * The field is the frozen field; if none is valid for the current step it is
 * refreshed first (scatter + field).  No thermostat force.
 * Errors: HPF_ERR_INVALID (which not in 1..3, F_out NULL with n > 0),
 * HPF_ERR_STATE, HPF_ERR_CUDA. */
hpf_status hpf_forces(hpf_ctx* ctx, float* F_out, int32_t which);

/* Advance n_steps steps (asynchronous).  With v the stored half-step
 * velocity, every step n does
 *   F = F_field(x_n) + F_bond(x_n) - gamma m v + sqrt(2 gamma m kT / dt) xi
 *   v <- v + dt F / m ;  x <- x + dt v
 * which is velocity-Verlet with its two half kicks merged.  xi = three
 * normals from Box-Muller on Philox4x32-10(counter = (tag, n lo, n hi, 0),
 * key = (seed lo, seed hi)), uniforms u = (2 (r >> 9) + 1) 2^-24; x, y from
 * (u0, u1) and z from (u2, u3).  The field is refreshed from the positions
 * when n % field_every == 0 (or when no field is valid) and held fixed in
 * between, as in the MD-SCF section.  With thermostat == 1 the step is the
 * Nose-Hoover scheme below instead (no friction or noise).  With thermostat
 * == 2 (Andersen, the section "MD methods and algorithms") there is no
 * friction or noise force; a bead collides at step n when the uniform of word
 * 0 of Philox4x32-10(counter = (tag, n lo, n hi, 1)) is below fl32(nu dt),
 * and then takes v <- sqrt(kT/m) xi + dt/(2m) F (xi as above): its on-step
 * velocity redrawn from the Maxwell distribution.  A launch that ends on a
 * refresh step deposits its final positions for that refresh.  Once
 * hpf_energy has been called on the state an hpf_step call ended at, later
 * calls' last launches also deposit their final positions (and, see
 * hpf_energy, form the observables' bead terms), until a call's deposit goes
 * unread before the next call; results do not depend on it.
 * Errors: HPF_ERR_INVALID (n_steps < 0), HPF_ERR_STATE, HPF_ERR_CUDA. */
hpf_status hpf_step(hpf_ctx* ctx, int32_t n_steps);

/* ---- Chain-partitioned runs ------------------------------------------------
 *
 * One system split into parts by whole chains, each part a context (for
 * example one per GPU).  The MD-SCF section drives every bead by one field of
 * the density of all beads, so at each refresh the parts' partial int64
 * meshes are summed (an exact, order-independent integer sum) and every part
 * computes the same field from the total; between refreshes the parts are
 * independent (bonds never cross parts, the field is frozen).
 *
 * hpf_set_tag_base: the part's beads are beads tag_base .. tag_base + n - 1
 * of the whole system; their noise counters (hpf_step) use those global tags,
 * so the parts draw the same noise as one context holding every chain.
 * Results stay indexed by the part's own tags 0 .. n - 1.  Any time after
 * hpf_init; tag_base >= 0 and tag_base + n_beads <= 2^24.
 * Errors: HPF_ERR_INVALID. */
hpf_status hpf_set_tag_base(hpf_ctx* ctx, int64_t tag_base);

/* hpf_step for one part: advances like hpf_step but returns where a field
 * refresh is due, with *steps_done the steps it ran and *mesh the device
 * address of the context's mesh ([S][Mz][My][Mx] int64, library-owned, valid
 * until the next call on the context) holding this part's own density of the
 * current positions.  The caller adds every other part's mesh into it (in
 * place, e.g. an all-reduce sum over the parts, ordered after the context's
 * stream and before the next call) and calls again: that call computes the
 * field from the mesh as it then stands and continues.  *mesh is NULL when the
 * call ran all n_steps before a refresh was due.  Sorting, bonds, angles,
 * dihedrals, the Langevin and Andersen thermostats and the fused deposit work
 * as in hpf_step, so parts driven this way with tag bases reproduce one
 * context's run bit for bit.  hpf_energy on a part gives its own beads'
 * kinetic and bonded terms and |P| and T of its beads; its field term is that
 * of the part's own density.  Asynchronous.
 * Errors: HPF_ERR_INVALID (n_steps < 0, NULL outputs, a Nose-Hoover context:
 * its thermostat couples every bead at every step), HPF_ERR_STATE, HPF_ERR_CUDA. */
hpf_status hpf_step_partial(hpf_ctx* ctx, int32_t n_steps, int32_t* steps_done, int64_t** mesh);

/* Observables at the current step, reduced in a fixed order (synchronises).
 * The bead terms are summed in float-float arithmetic over a grid set by n
 * alone (the bits do not depend on the GPU), except when the last hpf_step
 * call's final launch formed them itself: once calls are followed by the
 * observables of their end state, such a launch that does not end on a
 * refresh step (Langevin or no thermostat, bonds only, force_mode 0) forms
 * them from its final positions, and their order then follows the
 * persistent step grid (the SM count); either way the same quantities to
 * rounding.  Likewise such calls deposit their final positions, so the field
 * term needs no separate scatter.  Values:
 * out[0] kinetic energy of v_n = v_{n-1/2} + dt/(2m) F_n (F_n as in hpf_step;
 *   with Andersen, a bead colliding at step n counts its redrawn velocity),
 * out[1] bonded energy: bonds sum k (r - r0)^2 (float-float, ~1e-14 relative
 *   per bond), angles and dihedrals when set (FP64 per term),
 * out[2] field energy
 *   W = rho0 h^3 sum_nodes [1/2 kT sum_KK' chi phi_K phi_K' + 1/2 inv_kappa (sum phi - 1)^2]
 *   of a fresh scatter of the current positions, from exact 128-bit integer
 *   sums of the fixed-point densities over the nodes, combined once in FP64,
 * out[3] = out[0]+out[1]+out[2],
 * out[4] |total momentum| of v_n, out[5] kinetic temperature 2 KE / (3 N).
 * Errors: HPF_ERR_INVALID (out NULL), HPF_ERR_STATE, HPF_ERR_NONFINITE, HPF_ERR_CUDA. */
hpf_status hpf_energy(hpf_ctx* ctx, double out[6]);
/* hpf_energy in two halves: hpf_energy_start enqueues the kernels and the
 * copy of the six values (and of the kernels' error word) to pinned mirrors
 * on the context's stream and returns; hpf_energy_finish waits for those
 * copies only and returns the values of the step at which hpf_energy_start
 * was called, with the errors raised up to that point.  Work enqueued
 * between the two (hpf_upload_state, hpf_apply_state and hpf_step of the
 * next step) may still be running when it returns, so the next step's work
 * overlaps the host's reading of this one's; its errors surface at the next
 * synchronising call.  While a start is pending, hpf_energy, hpf_nh_conserved,
 * hpf_get_thermostat, hpf_set_thermostat, hpf_batch_energy and a second
 * hpf_energy_start return HPF_ERR_STATE.
 * Errors: as hpf_energy; HPF_ERR_STATE (hpf_energy_finish without a start). */
hpf_status hpf_energy_start(hpf_ctx* ctx);
hpf_status hpf_energy_finish(hpf_ctx* ctx, double out[6]);

/* Nose-Hoover NVT (thermostat == 1; the section "MD methods and algorithms"
 * names the thermostat for the canonical ensemble, with Hoover's equations
 *   dv/dt = F/m - xi v,  dxi/dt = (2K / (g kT) - 1) / tau^2,  deta/dt = xi,
 * g = 3 (n - 1) kinetic degrees of freedom (3 for n = 1)).  The state is
 * (x_n, v_{n-1/2}, xi, eta) with xi, eta at the middle of step n - 1.  Each
 * step n of hpf_step: the field refresh when due; F_n; v^E = v + dt/(2m) F_n;
 * two thermostat half steps T(dt/2) (the end of step n - 1, the start of step
 * n) on the kinetic energy K of v^E, each
 *   xi += (h/2) G(K); v *= exp(-xi h); K *= exp(-2 xi h); eta += xi h; xi += (h/2) G(K),
 *   G(K) = (2K / (g kT) - 1) / tau^2, h = dt/2;
 * then v <- v + dt/(2m) F_n; x <- x + dt v.  K is summed over the beads in
 * a fixed order in float-float arithmetic (pairs of FP32 numbers, about
 * 2^-45 relative per addition) and used in FP64.  hpf_energy reports the step's on-step quantities
 * after the pending half step (kinetic energy, |P| and T of s v^E).  Chains
 * of any length; not available in batches or learned windows.
 *
 * xi, eta of the state (out[2]); hpf_set_state resets them to zero.
 * Synchronises.  Errors: HPF_ERR_INVALID (no Nose-Hoover thermostat), HPF_ERR_CUDA. */
hpf_status hpf_get_thermostat(hpf_ctx* ctx, double out[2]);
/* Restore xi, eta (in[2], finite), e.g. with hpf_set_state from a checkpoint.
 * Synchronises.  Errors: HPF_ERR_INVALID, HPF_ERR_CUDA. */
hpf_status hpf_set_thermostat(hpf_ctx* ctx, const double in[2]);
/* The extended energy conserved by the Nose-Hoover equations at the current
 * step: the total energy of hpf_energy + g kT (tau^2 xi^2 / 2 + eta), with
 * xi, eta advanced by the pending half step.  Synchronises.
 * Errors: as hpf_energy, HPF_ERR_INVALID (no Nose-Hoover thermostat). */
hpf_status hpf_nh_conserved(hpf_ctx* ctx, double* H);

/* Stage profiling.  Every kernel launch of a context is counted by stage;
 * while profiling is enabled, CUDA events recorded on the context's stream
 * around each stage also accumulate its device time. */
#define HPF_STAGE_SCATTER 0 /* density scatter (+ mesh clear) */
#define HPF_STAGE_FIELD 1   /* field stencil */
#define HPF_STAGE_STEP 2    /* fused step kernel */
#define HPF_STAGE_SORT 3    /* bead sort */
#define HPF_STAGE_ENERGY 4  /* observables */
#define HPF_STAGE_OTHER 5   /* state load / unload, force output */
#define HPF_STAGE_COUNT 6

/* Turn event timing on (1) or off (0).  Errors: HPF_ERR_INVALID. */
hpf_status hpf_profile(hpf_ctx* ctx, int32_t enable);

/* Device milliseconds and kernel launches per stage since the last read
 * (either pointer may be NULL), then reset both.  Synchronises the stream.
 * Errors: HPF_ERR_INVALID, HPF_ERR_CUDA. */
hpf_status hpf_profile_read(hpf_ctx* ctx, double ms[HPF_STAGE_COUNT],
                            int64_t launches[HPF_STAGE_COUNT]);

/* ---- Batched replicas ----------------------------------------------------
 *
 * Many independent systems (for instance a chi scan of a phase diagram, each
 * replica with its own bead count, box, mesh and chi) advanced together.  The
 * paper runs one system per GPU; batching is this library's addition.  A
 * batch owns one hpf_ctx per replica, so every per-system call (set/get
 * state, forces, energy, density, field, order) works on a replica through
 * hpf_batch_replica.  hpf_batch_step advances all replicas with one batched
 * field launch and one persistent step launch per field period: the step
 * kernel's warps walk the segment lists of all replicas at once, so replicas
 * of 20k beads, which would fill a fraction of the GPU alone, share it.
 *
 * Requirements checked by hpf_batch_step (HPF_ERR_STATE otherwise): every
 * replica has a state, all replicas are at the same step, and all chains are
 * at most 64 beads (the warp-segment form); replicas with longer chains make
 * hpf_batch_step fall back to stepping the replicas one after another.
 * Requirements checked by hpf_batch_init (HPF_ERR_INVALID): 1 <= n_replicas
 * <= HPF_MAX_REPLICAS, equal n_species, field_every, sort_every and force_mode,
 * angles in all replicas or in none, and dihedrals in all or in none (their
 * constants may differ), and one thermostat, Langevin or Andersen, for all: the
 * batch runs one kernel form for all, and each replica's result is then the
 * bits of its own context. */
#define HPF_MAX_REPLICAS 64

typedef struct hpf_batch hpf_batch;

/* params: [n_replicas] parameter sets; stream as in hpf_init.
 * Errors: as hpf_init, plus HPF_ERR_INVALID for the batch requirements. */
hpf_status hpf_batch_init(const hpf_params* params, int32_t n_replicas, void* stream,
                          hpf_batch** out);

/* The context of replica r (owned by the batch; do not destroy it).  NULL if r is out of range. */
hpf_ctx* hpf_batch_replica(hpf_batch* batch, int32_t r);

/* Advance every replica by n_steps (asynchronous).  Each replica follows
 * exactly the same step as hpf_step on its own context would (same field
 * schedule, same Philox counters keyed by its own seed and tags), so the
 * results are those of R independent runs.  With graphs enabled (the
 * default), each pair of steady-state field periods is replayed from a CUDA
 * graph captured once per bead order.
 * Errors: HPF_ERR_INVALID (n_steps < 0), HPF_ERR_STATE, HPF_ERR_CUDA. */
hpf_status hpf_batch_step(hpf_batch* batch, int32_t n_steps);

/* Observables of every replica at its current step (hpf_energy's six values
 * each, out[n_replicas][6], replica order): all replicas' kernels are queued
 * on the batch's stream and the call synchronises once.  Errors: as
 * hpf_energy (the first failing replica's). */
hpf_status hpf_batch_energy(hpf_batch* batch, double* out);

/* Use CUDA graphs for steady-state periods (1, default) or plain launches (0). */
hpf_status hpf_batch_use_graphs(hpf_batch* batch, int32_t enable);

/* Free the batch and its replica contexts.  NULL is a no-op. */
hpf_status hpf_batch_destroy(hpf_batch* batch);

/* ---- Learned density propagator ------------------------------------------
 *
 * The paper has no counterpart to this part: it refreshes the density with a
 * CIC scatter at every field update.  Here a small 3-D convolutional network
 * predicts how the per-species volume fractions phi_K = rho_K / rho0 (the
 * quantities the external potential V_K of the MD-SCF section is built from)
 * change over K steps, so that between true scatters, taken every K steps,
 * the field can still be refreshed every step from predicted densities.
 *
 * Network (two species only): input x = (phi_A, phi_B at step t - K, phi_A,
 * phi_B at step t), 4 channels on the periodic Mx x My x Mz mesh, whose input
 * channels are formed in FP32 as (s (phi(t) - phi(t - K)), phi(t)) per
 * species before the BF16 rounding, s the handle's change scale; three 3x3x3
 * periodic convolutions (cross-correlation) 4 -> 16 -> 16 -> 2 channels
 * with SiLU after the first two; output dphi = (last layer) / s = predicted
 * phi(t + K) - phi(t).  The scale s brings density changes (about 1e-2 per
 * step) to order one in the network's units, so the weights that read them
 * need not be far larger than their initial values.
 * A convolution computes out[co](n) = b[co] + sum_d sum_ci W[d][ci][co]
 * in[ci](n + d) over the 27 offsets d = (dz, dy, dx) in {-1, 0, 1}^3, z-major.
 * Weights and activations are BF16 on the tensor cores with FP32
 * accumulation (forward and data gradients on tcgen05 with tensor-memory
 * accumulators; the forward convolutions are persistent, one CTA per SM
 * sweeping columns of the mesh along z); the master parameters and Adam
 * state are FP32.  The
 * tensor-core waits are bounded: one that gives up makes the next call that
 * synchronises return HPF_ERR_TIMEOUT (once).
 *
 * Parameter vector (hpf_prop_param_count() floats): for each layer in order,
 * W [27][C_in][C_out] then b [C_out].  Mesh arrays are planar FP32,
 * [channel][Mz][My][Mx].  Pointers may be host or device memory.
 * The network's buffers belong to the handle: use one handle from one
 * stream at a time (hpf_step_learned runs it on the context's stream). */
typedef struct hpf_prop hpf_prop;

/* mesh = (Mx, My, Mz), each 2..1024, at most 2^26 nodes; stream as in
 * hpf_init.  The weights start at zero (the network predicts no change).
 * Errors: HPF_ERR_INVALID, HPF_ERR_NOMEM, HPF_ERR_CUDA. */
hpf_status hpf_prop_init(const int32_t mesh[3], void* stream, hpf_prop** out);
hpf_status hpf_prop_destroy(hpf_prop* prop); /* NULL is a no-op */
int32_t hpf_prop_param_count(void);

/* The change scale s (default 1): > 0 and finite, else HPF_ERR_INVALID.  It
 * is not part of the parameter vector; set it before training and keep it
 * with the weights. */
hpf_status hpf_prop_set_scale(hpf_prop* prop, float scale);
hpf_status hpf_prop_get_scale(const hpf_prop* prop, float* scale);

/* Self-test of the forward convolutions' bounded waits: the first layer runs
 * on the handle's current input with its finished output planes never
 * signalled, so every CTA's waits run out (0.2 s), raise the timeout flag,
 * end every role of the CTA and release its tensor memory.  The flag is
 * cleared again, so the handle stays usable; *seconds (may be NULL) is the
 * host-measured time.  Returns HPF_ERR_TIMEOUT when the waits gave up as
 * designed, HPF_OK if they did not act.  Synchronises.
 * Errors: HPF_ERR_INVALID, HPF_ERR_CUDA. */
hpf_status hpf_prop_selftest_timeout(hpf_prop* prop, double* seconds);

/* At most ctas CTAs for the persistent forward convolutions (the output
 * planes are split evenly over them); 0 restores the default of two CTAs per
 * SM.  Results do not depend on it (bit for bit).  Errors: HPF_ERR_INVALID
 * (ctas < 0). */
hpf_status hpf_prop_set_ctas(hpf_prop* prop, int32_t ctas);

/* Load [param_count] FP32 parameters (and reset Adam); synchronises. */
hpf_status hpf_prop_set_weights(hpf_prop* prop, const float* params);
/* Copy the FP32 parameters out (synchronises for a host destination). */
hpf_status hpf_prop_get_weights(hpf_prop* prop, float* params);

/* dphi [2][Mz][My][Mx] = network(x [4][Mz][My][Mx]).  Arrays on the current
 * device are read and written in place by the kernels on the handle's
 * stream (x is consumed by the first kernel, so it may alias dphi; neither
 * may change until the stream has passed the call); host arrays go through
 * the handle's staging buffers.  Synchronises for a host destination (and
 * then reports HPF_ERR_TIMEOUT as above); with a device destination it
 * returns without waiting.  Errors: HPF_ERR_INVALID (NULL), HPF_ERR_CUDA. */
hpf_status hpf_prop_forward(hpf_prop* prop, const float* x, float* dphi);

/* Autoregressive use of a network trained at lag 1 (the per-step variant of
 * the propagator): from x = (phi(t - 1), phi(t)) [4][Mz][My][Mx], steps times
 * phi(t + 1) = phi(t) + network(phi(t - 1), phi(t)), each prediction fed
 * back as the next input (FP32 sums); phi_out [2][Mz][My][Mx] = the predicted
 * phi(t + steps).  With a network trained at lag L and steps = 1 it is that
 * network's prediction phi(t) + dphi.  Synchronises for a host destination.
 * Errors: HPF_ERR_INVALID (steps < 1, NULL), HPF_ERR_CUDA, HPF_ERR_TIMEOUT. */
hpf_status hpf_prop_rollout(hpf_prop* prop, const float* x, int32_t steps, float* phi_out);

/* Loss L = mean over the 2 x M outputs of (s network(x) - s (phi_next - x[2:4]))^2,
 * i.e. s^2 times the mean squared error of the predicted change,
 * and its gradient with respect to the parameter vector (back-propagation
 * through the same BF16 kernels: data gradients with flipped, transposed
 * weights, weight gradients as tensor-core voxel reductions).  phi_next is
 * [2][Mz][My][Mx]; grads [param_count] and loss may be NULL.  Synchronises
 * when loss is given or grads is host memory. */
hpf_status hpf_prop_backward(hpf_prop* prop, const float* x, const float* phi_next, float* grads,
                             double* loss);

/* One Adam update (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) of the
 * parameters with the given gradient vector.  Errors: HPF_ERR_INVALID (lr <= 0). */
hpf_status hpf_prop_adam_step(hpf_prop* prop, const float* grads, float lr);

/* hpf_prop_backward followed by hpf_prop_adam_step with its own gradients,
 * all on the device (the loss before the update is returned when loss is not
 * NULL, which synchronises). */
hpf_status hpf_prop_train_step(hpf_prop* prop, const float* x, const float* phi_next, float lr,
                               double* loss);

/* phi [n_species][Mz][My][Mx] FP32 of the context's current positions: the
 * CIC density mesh times 2^-39 / (rho0 h^3).  Errors: HPF_ERR_STATE, HPF_ERR_CUDA. */
hpf_status hpf_density_phi(hpf_ctx* ctx, float* phi);

/* Field-force error of a candidate density at the current positions:
 * eps = || F(phi) - F(true) ||_2 / || F(true) ||_2 over all beads and
 * components, where F(true) is the field force of the true CIC density and
 * F(phi) that of the candidate phi [n_species][Mz][My][Mx] (FP32, taken to
 * the mesh's fixed point; negative values count as zero).  Leaves the field
 * of the true density in force.  Synchronises.
 * Errors: HPF_ERR_INVALID, HPF_ERR_STATE, HPF_ERR_CUDA. */
hpf_status hpf_judge_density(hpf_ctx* ctx, const float* phi, double* eps);

/* The smoothed-density study (the propagator's accuracy question of the
 * learned part; the paper has no counterpart): a periodic binomial filter of
 * phi meshes and a judge between two densities.
 *
 * hpf_smooth_phi: phi_out = the filter (1/4, 1/2, 1/4) applied along x, y and
 * z in turn, `passes` times (0..64; variance passes/2 cells^2 per axis), to
 * phi_in [n_species][Mz][My][Mx] FP32 (periodic; host or device; phi_out may
 * equal phi_in).  Synchronises for a host destination.
 * hpf_judge_density_pair: eps = || F(phi_cand) - F(phi_ref) ||_2 /
 * || F(phi_ref) ||_2, the field forces (trilinear gather of the
 * central-difference gradient, as the judge of hpf_step_learned) of the two
 * densities at the current positions, each taken to the mesh's fixed point
 * (negative values count as zero).  Leaves the field of the true density in
 * force.  Synchronises.
 * Errors: HPF_ERR_INVALID, HPF_ERR_STATE, HPF_ERR_CUDA. */
hpf_status hpf_smooth_phi(hpf_ctx* ctx, const float* phi_in, float* phi_out, int32_t passes);
hpf_status hpf_judge_density_pair(hpf_ctx* ctx, const float* phi_cand, const float* phi_ref,
                                  double* eps);

/* How hpf_step_learned runs an accepted-form (learned) window.  in_launch = 1
 * (the default): one step-kernel launch for the whole window, the field at
 * window step j being (1 - j/K) F(D(t)) + (j/K) F(D(t) + dphi), F the field of
 * a mesh -- the field of D(t) + (j/K) dphi, since the field is linear in the
 * density -- with both cells' polynomials cached per bead (contexts whose
 * chains fit warp segments and with force_mode 0; others run per step).
 * in_launch = 0: one launch per step on the field of the integer mesh
 * D(t) + (j/K) dphi (in the mesh's fixed point) refreshed every step.  The two
 * agree to FP32 rounding.  Errors: HPF_ERR_INVALID, HPF_ERR_NOMEM. */
hpf_status hpf_learned_mode(hpf_ctx* ctx, int32_t in_launch);

/* Outcome of hpf_step_learned (totals of the call). */
typedef struct {
    int64_t steps;    /* steps advanced */
    int32_t windows;  /* windows of K steps completed */
    int32_t learned;  /* windows run on predicted densities and accepted */
    int32_t rejected; /* learned windows whose judged error exceeded tol: rolled back, re-run plain */
    int32_t plain;    /* windows run plain from the start (no history yet, or after a rejection) */
    int32_t judged;   /* predictions judged (learned and shadow) */
    double eps_last;  /* last judged field-force error */
    double eps_max;   /* largest judged error */
    double eps_sum;   /* sum of judged errors */
} hpf_learned_stats;

/* Advance n_windows windows of K steps (K in 2..64) with the learned
 * propagator (two species; the network's mesh must equal the context's).
 * A window starts at a true update t: the density D(t) is scattered and the
 * field refreshed from it.  A learned window predicts dphi = network(phi(t-K),
 * phi(t)) and runs steps t+1 .. t+K-1 on the field of D(t) + (j/K) dphi (in
 * the mesh's fixed point); the last step scatters the true D(t+K).  There the
 * judge computes eps (as hpf_judge_density) between the field force of the
 * predicted D(t) + dphi and of the true D(t+K).  eps <= tol accepts the
 * window; otherwise the state at t is restored and the window re-run with a
 * true scatter and field refresh every step (the plain update), and the next
 * windows run plain while their predictions are judged in the shadow, until
 * one meets tol.  After a rejection or a failed shadow judgement the next
 * 1, 2, 4, ... (at most 64) plain windows skip the prediction and the judge,
 * so a network that keeps failing costs little.  The first window of a
 * context runs plain (it builds the phi(t-K) history).  Beads are re-sorted
 * only at window starts.  With zero network weights a learned window equals
 * field_every = K exactly.
 * Synchronises once per window.  stats may be NULL.
 * Errors: HPF_ERR_INVALID, HPF_ERR_STATE, HPF_ERR_CUDA, HPF_ERR_NONFINITE,
 * HPF_ERR_OVERFLOW. */
hpf_status hpf_step_learned(hpf_ctx* ctx, hpf_prop* prop, int32_t n_windows, int32_t K, double tol,
                            hpf_learned_stats* stats);

/* ---- Field forces without any device allocation ---------------------------
 *
 * The paper has no counterpart to this entry point.  It is here for callers
 * that cannot let a library allocate GPU memory: for example a host program
 * whose own memory pool has already reserved nearly all of the device, or a
 * program that must not pay the device-wide synchronisation that cudaMalloc
 * and cudaFree can cause in the middle of its work.  Such a caller owns every
 * buffer it passes; the library's own working memory (one int64 density mesh
 * and the float4 field) is a single file-scope static __device__
 * array of HPF_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads this
 * library holds until the process exits.
 *
 * The call computes, with no context, the field force that hpf_forces gives
 * with HPF_FORCE_FIELD right after loading these positions: CIC scatter of the
 * beads, V and grad V of that mesh, trilinear gather -grad V_T at every bead.
 * Only n_species, mesh, box, kT, rho0, inv_kappa and chi of `params` are used
 * (the force is always the interpolated-gradient one, force_mode 0).
 *   pos   [n][3] float32 positions, device memory of the current device
 *   type  [n]    int32 species; a species outside [0, n_species) gets a NaN
 *                force and adds nothing to the density
 *   F_out [n][3] float32 output, device memory of the current device
 *   stream       cudaStream_t the kernels are enqueued on (NULL: legacy
 *                default stream); the call returns without waiting
 * The first call on a device looks up the scratch's device address (with
 * cudaGetSymbolAddress, that device current) and caches it; make that first
 * call before any stream capture.  All calls on one device share the
 * scratch, and it keeps the previous call's contents (each call clears the
 * density mesh it needs itself): calls that overlap on the GPU (two streams
 * or threads without ordering between them) race and give wrong forces, so
 * order them, for instance on one stream.
 * Errors: HPF_ERR_INVALID (a field parameter hpf_init would refuse, n outside
 * [0, HPF_MAX_BEADS], or with n > 0 a NULL pointer, a host pointer or one to
 * another GPU's memory), HPF_ERR_SCRATCH (the mesh needs more than
 * HPF_NOALLOC_SCRATCH_BYTES; see hpf_noalloc_scratch_bytes), HPF_ERR_CUDA. */
#define HPF_NOALLOC_SCRATCH_BYTES (32u << 20) /* 32 MiB: fits a 70^3 mesh of up to 3 species */

/* Scratch bytes hpf_field_forces_noalloc needs for these parameters (0 if the
 * species count or mesh is invalid). */
size_t hpf_noalloc_scratch_bytes(const hpf_params* params);

hpf_status hpf_field_forces_noalloc(const hpf_params* params, const float* pos,
                                    const int32_t* type, int32_t n, float* F_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HPF_H */
