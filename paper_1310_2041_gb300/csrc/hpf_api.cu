// hpf_api.cu -- the C ABI declared in include/hpf.h: context, state, schedule.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "hpf_internal.cuh"
#include "nh_internal.cuh"

using namespace hpf;

struct hpf_ctx {
    hpf_params p;
    cudaStream_t stream = nullptr;
    int n = 0, S = 0;
    MeshGeom geom{};
    StepConsts sc{};
    FieldCoef coef{};
    EnergyConsts ec{};
    float* state_mem = nullptr;     // 2 x 6 x n floats
    StateBuf st[2]{};
    int cur = 0;
    uint32_t* meta = nullptr;
    uint32_t* meta2 = nullptr;        // sort target
    SortBufs sb{};
    void* sort_mem = nullptr;
    int C = 0;                        // number of chains
    int max_chain = 0;                // longest chain (beads)
    bool warp_mode = false;           // chains fit warp segments: barrier-free step kernel
    long long last_sort_step = 0;
    unsigned long long* D = nullptr;  // two int64 density meshes, [2][S][M]
    int dmesh = 0;                    // which one is the context's mesh
    long long mesh_step = -1;         // step whose positions it holds (-1: none / injected)
    bool next_zero = false;           // the other mesh is known to be all zero
    long long part_step = -1;         // step whose partial mesh hpf_step_partial handed out
    // deposit at the end of hpf_step calls: switched on when the observables
    // of a step's final state had to scatter it, off again when such a
    // deposit was not used before the next call
    bool want_end_mesh = false;
    bool end_mesh_unused = false;     // the last call's end deposit is still unread
    long long end_of_call_step = -1;  // the step the last hpf_step call ended on
    // observables' bead partials formed by the step launch that ended at
    // obs_step (k_step_warp_obs), obs_nb CTAs' worth
    float2* obs_part = nullptr;
    long long obs_step = -1;
    int obs_nb = 0;
    float4* G = nullptr;              // field mesh (ghosted)
    float4* field_stage = nullptr;    // dense copy of the field for hpf_field's output
    FieldCoef* d_coef = nullptr;      // the stencil coefficients in device memory
    int field_tile = -1;              // tiled stencil shape chosen by the autotuner (-1: not yet)
    int tmap_tile = -1;               // tile the tensor maps below were encoded for
    bool tmap_ok = false;             // TMA usable for this mesh
    CUtensorMap tmap[2];              // over mesh buffers 0 and 1
    float* out_f = nullptr;           // 2 x 3n floats of tag-order output staging
    void* stage = nullptr;            // set_state input staging
    int* dflag = nullptr;             // [0] kernel flags, [1..4] validation counters
    int* hflag = nullptr;             // pinned mirror
    double* partials = nullptr;
    double* d_out6 = nullptr;
    double* h_out6 = nullptr;         // pinned
    bool has_state = false;
    bool field_valid = false;
    long long step = 0;
    long long field_step = -1;
    // profiling: kernel launches per stage, and event pairs while enabled
    bool profiling = false;
    long long launches[HPF_STAGE_COUNT] = {};
    struct EvPair {
        cudaEvent_t a, b;
        int stage;
    };
    std::vector<EvPair> ev_used;
    std::vector<cudaEvent_t> ev_free;
    std::string err;
    struct LearnedBufs* learned = nullptr;  // learned-propagator buffers (allocated on first use)
    // Nose-Hoover (thermostat == 1): device state and partials, the stored
    // force (two buffers of [3][n]), constants, host mirror
    NhDev* nh = nullptr;
    double* nh_part = nullptr;
    float* nh_F = nullptr;
    int nh_f = 0;  // force buffer written last
    NhConsts nhc{};
    double* h_nh = nullptr;  // pinned [2]: xi, eta
    // pipelined uploads (hpf_upload_state / hpf_apply_state): two staging
    // slots of [6n] floats, the context's copy stream, and per slot the event
    // of its copy and the event of the permutation that last read it
    float* up_stage[2] = {nullptr, nullptr};
    cudaStream_t up_stream = nullptr;
    cudaEvent_t up_done[2] = {nullptr, nullptr};
    cudaEvent_t up_free[2] = {nullptr, nullptr};
    int up_slot = 0;
    bool up_ready = false;    // stream, events and both slots exist
    bool up_pending = false;
    bool energy_pending = false;  // hpf_energy_start issued, hpf_energy_finish not yet
    cudaEvent_t energy_ev = nullptr;  // after hpf_energy_start's copies to the host
};

// Buffers of the learned-propagator driver and the density judge.
struct LearnedBufs {
    unsigned long long* Dbase = nullptr;  // D(t) at the window start [S][M]
    unsigned long long* Dp = nullptr;     // predicted / candidate mesh [S][M]
    CUtensorMap tmap;                     // over Dp
    int tmap_tile = -1;
    bool tmap_ok = false;
    float* x = nullptr;     // network input [max(4, S)][M]: phi(t - K), phi(t)
    float* dphi = nullptr;  // predicted change [S][M]
    float* snap = nullptr;  // state at the window start [6][n]
    double* acc = nullptr;  // judge sums [2] and their partials
    double* h_acc = nullptr;
    long long hist_step = -1;  // step whose phi is in x[0:2] (-1: none)
    bool plain_mode = false;   // run plain windows (shadow-judged) until a prediction meets tol
    int backoff = 0;           // plain windows to skip between shadow judgements (doubles per failure)
    int skip_left = 0;         // plain windows left before the next shadow judgement
    float4* G2 = nullptr;      // field of the window's predicted end density (ghosted)
    bool in_launch = true;     // a learned window in one launch (interpolated fields)
};

namespace {

hpf_status fail(hpf_ctx* c, hpf_status s, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define CUDA_TRY(ctx, call)                                                                    \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? HPF_ERR_NOMEM : HPF_ERR_CUDA, \
                        "%s: %s", #call, cudaGetErrorString(e_));                              \
    } while (0)

#define LAUNCH_CHECK(ctx)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = cudaGetLastError();                                                   \
        if (e_ != cudaSuccess)                                                                 \
            return fail((ctx), HPF_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e_));     \
    } while (0)

cudaEvent_t take_event(hpf_ctx* c) {
    if (!c->ev_free.empty()) {
        cudaEvent_t e = c->ev_free.back();
        c->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Counts the kernels of one stage and, while profiling, brackets them with
// events on the context's stream.
struct StageScope {
    hpf_ctx* c;
    int stage, kernels;
    cudaEvent_t a = nullptr;
    StageScope(hpf_ctx* c_, int stage_, int kernels_) : c(c_), stage(stage_), kernels(kernels_) {
        if (c->profiling && (a = take_event(c)) != nullptr) cudaEventRecord(a, c->stream);
    }
    ~StageScope() {
        c->launches[stage] += kernels;
        if (!a) return;
        cudaEvent_t b = take_event(c);
        if (!b) return;
        cudaEventRecord(b, c->stream);
        c->ev_used.push_back({a, b, stage});
    }
};

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy to a caller pointer; wait for the copy when the destination is host memory.
hpf_status copy_out(hpf_ctx* c, void* dst, const void* src, size_t bytes) {
    if (!dst || bytes == 0) return HPF_OK;
    CUDA_TRY(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
    if (!is_device_ptr(dst)) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return HPF_OK;
}

}  // namespace

// The mesh and field parameters (shared with the allocation-free entry point).
hpf_status hpf::validate_field_params(const hpf_params* p) {
    if (!p) return HPF_ERR_INVALID;
    if (p->n_species < 1 || p->n_species > HPF_MAX_SPECIES) return HPF_ERR_INVALID;
    for (int a = 0; a < 3; ++a) {
        if (p->mesh[a] < 2 || p->mesh[a] > 4096) return HPF_ERR_INVALID;
        if (!(p->box[a] > 0.0f) || !isfinite(p->box[a])) return HPF_ERR_INVALID;
    }
    if ((long long)(p->mesh[0] + 1) * (p->mesh[1] + 1) * (p->mesh[2] + 1) * p->n_species >
        (1LL << 31) - 1)
        return HPF_ERR_INVALID;
    if (!(p->rho0 > 0) || !(p->kT >= 0) || !isfinite(p->kT) || !isfinite(p->inv_kappa))
        return HPF_ERR_INVALID;
    for (int k = 0; k < p->n_species; ++k)
        for (int j = 0; j < p->n_species; ++j) {
            const double a = p->chi[k * HPF_MAX_SPECIES + j], b = p->chi[j * HPF_MAX_SPECIES + k];
            if (!isfinite(a) || a != b) return HPF_ERR_INVALID;  // chi must be symmetric
        }
    return HPF_OK;
}

namespace {

hpf_status validate_params(const hpf_params* p) {
    if (!p) return HPF_ERR_INVALID;
    if (p->n_beads < 0) return HPF_ERR_INVALID;
    if (p->n_beads > HPF_MAX_BEADS) return HPF_ERR_OVERFLOW;
    const hpf_status f = validate_field_params(p);
    if (f != HPF_OK) return f;
    if (!(p->mass > 0) || !(p->dt > 0) || !(p->gamma >= 0)) return HPF_ERR_INVALID;
    if (!isfinite(p->bond_k) || !isfinite(p->bond_r0)) return HPF_ERR_INVALID;
    if (p->field_every < 1 || p->sort_every < 0) return HPF_ERR_INVALID;
    if (p->force_mode < 0 || p->force_mode > 2) return HPF_ERR_INVALID;
    if (!isfinite(p->angle_k) || !(p->angle_cos0 >= -1.0 && p->angle_cos0 <= 1.0))
        return HPF_ERR_INVALID;
    if (p->angle_form < 0 || p->angle_form > 1 ||
        (p->angle_form == 1 && !(p->angle_theta0 >= 0.0 && p->angle_theta0 <= M_PI)))
        return HPF_ERR_INVALID;
    if (!isfinite(p->dihedral_k) || !isfinite(p->dihedral_delta) ||
        (p->dihedral_k != 0.0 && (p->dihedral_n < 1 || p->dihedral_n > 6)))
        return HPF_ERR_INVALID;
    if (p->thermostat < 0 || p->thermostat > 2) return HPF_ERR_INVALID;
    if (p->thermostat == 2 && !(p->andersen_nu >= 0.0 && isfinite(p->andersen_nu)))
        return HPF_ERR_INVALID;
    if (p->thermostat == 1 && !(p->nh_tau > 0.0 && isfinite(p->nh_tau))) return HPF_ERR_INVALID;
    return HPF_OK;
}

void derive_constants(hpf_ctx* c) {
    const hpf_params& p = c->p;
    MeshGeom& g = c->geom;
    g.mx = p.mesh[0];
    g.my = p.mesh[1];
    g.mz = p.mesh[2];
    g.nodes = g.mx * g.my * g.mz;
    g.gx = g.mx + 1;
    g.gxy = (g.mx + 1) * (g.my + 1);
    g.gnodes = g.gxy * (g.mz + 1);
    double h[3], vol = 1.0;
    for (int a = 0; a < 3; ++a) {
        g.inv_h[a] = (float)((double)p.mesh[a] / (double)p.box[a]);
        g.inv_m[a] = 1.0f / (float)p.mesh[a];
        h[a] = (double)p.box[a] / (double)p.mesh[a];
        vol *= h[a];
    }
    const double phi_c = ldexp(1.0, -3 * HPF_FRAC_BITS) / (p.rho0 * vol);
    FieldCoef& f = c->coef;
    memset(&f, 0, sizeof f);
    f.S = p.n_species;
    f.v0 = (float)(-p.inv_kappa);
    for (int k = 0; k < p.n_species; ++k)
        for (int j = 0; j < p.n_species; ++j) {
            const double A = p.kT * p.chi[k * HPF_MAX_SPECIES + j] + p.inv_kappa;
            f.gx[k][j] = (float)(A * phi_c / (2.0 * h[0]));
            f.gy[k][j] = (float)(A * phi_c / (2.0 * h[1]));
            f.gz[k][j] = (float)(A * phi_c / (2.0 * h[2]));
            f.v[k][j] = (float)(A * phi_c);
        }
    StepConsts& s = c->sc;
    s.dt = (float)p.dt;
    s.dt_m = (float)(p.dt / p.mass);
    // Nose-Hoover and Andersen replace the Langevin friction and noise
    const double gamma = p.thermostat == 0 ? p.gamma : 0.0;
    s.fric = (float)(gamma * p.mass);
    s.sigma = (float)sqrt(2.0 * gamma * p.mass * p.kT / p.dt);
    s.two_k = (float)(2.0 * p.bond_k);
    s.r0 = (float)p.bond_r0;
    s.seed_lo = (uint32_t)p.seed;
    s.seed_hi = (uint32_t)(p.seed >> 32);
    for (int r = 0; r < 10; ++r) {
        s.rk0[r] = s.seed_lo + (uint32_t)r * 0x9E3779B9u;
        s.rk1[r] = s.seed_hi + (uint32_t)r * 0xBB67AE85u;
    }
    s.force_mode = p.force_mode;
    s.two_ka = (float)(2.0 * p.angle_k);
    s.cos0 = (float)p.angle_cos0;
    s.angle_form = p.angle_form;
    s.th0 = (float)p.angle_theta0;
    s.p_coll = p.thermostat == 2 ? (float)(p.andersen_nu * p.dt) : 0.0f;
    s.sig_v = (float)sqrt(p.kT / p.mass);
    s.kd = (float)p.dihedral_k;
    s.nd = p.dihedral_k != 0.0 ? p.dihedral_n : 1;
    s.cd = (float)cos(p.dihedral_delta);
    s.sd = (float)sin(p.dihedral_delta);
    EnergyConsts& e = c->ec;
    memset(&e, 0, sizeof e);
    e.half_dt_m = 0.5 * p.dt / p.mass;
    e.mass = p.mass;
    e.bond_k = p.bond_k;
    e.r0 = p.bond_r0;
    e.r0_hi = (float)p.bond_r0;
    e.r0_lo = (float)(p.bond_r0 - (double)e.r0_hi);
    e.bond_k_hi = (float)p.bond_k;
    e.bond_k_lo = (float)(p.bond_k - (double)e.bond_k_hi);
    e.kT = p.kT;
    e.angle_k = p.angle_k;
    e.cos0 = p.angle_cos0;
    e.angle_form = p.angle_form;
    e.theta0 = p.angle_theta0;
    e.dih_k = p.dihedral_k;
    e.dih_n = p.dihedral_k != 0.0 ? p.dihedral_n : 1;
    e.dih_cd = cos(p.dihedral_delta);
    e.dih_sd = sin(p.dihedral_delta);
    e.inv_kappa = p.inv_kappa;
    e.phi_c = phi_c;
    e.w_scale = p.rho0 * vol;
    for (int k = 0; k < p.n_species; ++k)
        for (int j = 0; j < p.n_species; ++j) e.chi[k][j] = p.chi[k * HPF_MAX_SPECIES + j];
    e.S = p.n_species;
    e.n = p.n_beads;
    NhConsts& t = c->nhc;
    t.h = 0.5 * p.dt;
    t.dof_kT = (p.n_beads > 1 ? 3.0 * (p.n_beads - 1) : 3.0 * p.n_beads) * p.kT;
    t.two_over_dof_kT = t.dof_kT > 0.0 ? 2.0 / t.dof_kT : 0.0;
    t.inv_tau2 = p.thermostat == 1 ? 1.0 / (p.nh_tau * p.nh_tau) : 0.0;
    t.mass = p.mass;
}

size_t stage_bytes(int n) {
    // pos, vel [3n] f32; type [n] i32; bonds [2n] i32 (a chain set has < n bonds)
    return (size_t)n * (3 + 3 + 1 + 2) * 4 + 256;
}

StateBuf& cur_state(hpf_ctx* c) { return c->st[c->cur]; }

size_t mesh_words(const hpf_ctx* c) { return (size_t)c->geom.nodes * c->S; }
unsigned long long* mesh_buf(hpf_ctx* c, int k) { return c->D + (size_t)k * mesh_words(c); }

// Tensor maps of both mesh buffers for a tile shape (TMA box = tile + halo).
void ensure_tmaps(hpf_ctx* c, int tile) {
    if (c->tmap_tile == tile) return;
    c->tmap_ok = c->S <= 4;
    for (int k = 0; k < 2 && c->tmap_ok; ++k)
        c->tmap_ok = make_mesh_tensor_map(&c->tmap[k], reinterpret_cast<const long long*>(mesh_buf(c, k)),
                                          c->geom, c->S, tile);
    c->tmap_tile = tile;
}

// One replica's record of the tiled stencil reading mesh D (tensor map tm,
// usable when tm_ok) and clearing D_clear (may be NULL).
void fill_field_rep_mesh(hpf_ctx* c, int tile, const unsigned long long* D, const CUtensorMap& tm,
                         bool tm_ok, unsigned long long* D_clear, TiledFieldRep& fr, int& blocks) {
    fr.tmap = tm;
    fr.coef = c->d_coef;
    fr.g = c->geom;
    fr.D = reinterpret_cast<const long long*>(D);
    fr.G = c->G;
    fr.D_clear = D_clear;
    fr.use_tma = tm_ok ? 1 : 0;
    int nb = 0;
    tile_grid(c->geom, tile, &fr.tiles_x, &fr.tiles_y, &nb);
    fr.blk_begin = blocks;
    blocks += nb;
}

// The record reading mesh buffer `dm` and clearing the other one.
void fill_field_rep(hpf_ctx* c, int tile, int dm, TiledFieldRep& fr, int& blocks) {
    ensure_tmaps(c, tile);
    fill_field_rep_mesh(c, tile, mesh_buf(c, dm), c->tmap[dm], c->tmap_ok, mesh_buf(c, dm ^ 1), fr,
                        blocks);
}

// Time every candidate tile on this launch shape and keep the fastest.  The
// candidates compute the same field (the last launch leaves it in place).
template <class Params, class Fill>
int autotune_tile(cudaStream_t s, int S, Fill fill) {
    if (S > 4) return -1;
    // Each candidate timed launch by launch (an event between launches, so
    // what counts is a launch's own duration, as in a step loop where the
    // next kernel waits on the field), the median of kReps launches per
    // round, the best of kRounds interleaved rounds (a single timing of a few
    // launches picked a 1.5x slower tile often enough to matter).
    constexpr int kRounds = 3, kReps = 5;
    cudaEvent_t ev[kReps + 1];
    int made = 0;
    for (; made <= kReps; ++made)
        if (cudaEventCreate(&ev[made]) != cudaSuccess) break;
    if (made <= kReps) {
        for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
        cudaGetLastError();
        return 0;
    }
    const int cands = field_tile_candidates();
    std::vector<float> score(cands, 1e30f);
    for (int round = 0; round < kRounds; ++round) {
        for (int t = 0; t < cands; ++t) {
            Params p;
            fill(t, p);
            launch_field_tiled(p, S, t, s);  // warm
            cudaEventRecord(ev[0], s);
            for (int rep = 0; rep < kReps; ++rep) {
                launch_field_tiled(p, S, t, s);
                cudaEventRecord(ev[rep + 1], s);
            }
            if (cudaEventSynchronize(ev[kReps]) != cudaSuccess) continue;
            float d[kReps];
            bool ok = true;
            for (int rep = 0; rep < kReps; ++rep)
                ok = ok && cudaEventElapsedTime(&d[rep], ev[rep], ev[rep + 1]) == cudaSuccess;
            if (!ok) continue;
            std::sort(d, d + kReps);
            score[t] = std::min(score[t], d[kReps / 2]);
        }
    }
    int best = 0;
    for (int t = 1; t < cands; ++t)
        if (score[t] < score[best]) best = t;
    cudaGetLastError();
    for (int k = 0; k <= kReps; ++k) cudaEventDestroy(ev[k]);
    return best;
}

// The context's mesh holds the density of the current positions afterwards:
// scatter into the other buffer (cleared first unless known zero) and flip.
hpf_status scatter_current(hpf_ctx* c) {
    if (c->mesh_step == c->step) {
        c->end_mesh_unused = false;
        return HPF_OK;
    }
    unsigned long long* dst = mesh_buf(c, c->dmesh ^ 1);
    {
        StageScope sc(c, HPF_STAGE_SCATTER, c->n > 0 ? 1 : 0);
        if (!c->next_zero)
            CUDA_TRY(c, cudaMemsetAsync(dst, 0, sizeof(unsigned long long) * mesh_words(c),
                                        c->stream));
        launch_scatter(cur_state(c), c->meta, c->n, c->geom, dst, c->stream);
    }
    LAUNCH_CHECK(c);
    c->dmesh ^= 1;
    c->mesh_step = c->step;
    c->next_zero = false;
    return HPF_OK;
}

// Field of the context's mesh; the kernel also clears the other mesh, the
// target of the next scatter.
hpf_status run_field(hpf_ctx* c) {
    if (c->S <= 4) {
        // the tiled (TMA-staged) stencil with one replica; a batch runs the same
        // kernel, so contexts and batch members agree bit for bit
        if (c->field_tile < 0)
            c->field_tile = autotune_tile<SingleFieldParams>(c->stream, c->S, [&](int t, SingleFieldParams& p) {
                memset(&p, 0, sizeof p);
                p.R = 1;
                p.flag = c->dflag;
                fill_field_rep(c, t, c->dmesh, p.rep[0], p.blocks);
            });
        StageScope sc(c, HPF_STAGE_FIELD, 1);
        SingleFieldParams p;
        memset(&p, 0, sizeof p);
        p.R = 1;
        p.flag = c->dflag;
        fill_field_rep(c, c->field_tile, c->dmesh, p.rep[0], p.blocks);
        launch_field_tiled(p, c->S, c->field_tile, c->stream);
    } else {
        StageScope sc(c, HPF_STAGE_FIELD, 1);
        BatchFieldParams fp;
        memset(&fp, 0, sizeof fp);
        fp.R = 1;
        fp.coef = c->d_coef;
        fp.rep[0].g = c->geom;
        fp.rep[0].D = reinterpret_cast<const long long*>(mesh_buf(c, c->dmesh));
        fp.rep[0].G = c->G;
        fp.rep[0].D_clear = mesh_buf(c, c->dmesh ^ 1);
        fp.rep[0].blk_begin = 0;
        fp.blocks = (c->geom.gnodes + 255) / 256;
        launch_field_batch(fp, c->S, c->stream);
    }
    LAUNCH_CHECK(c);
    c->next_zero = true;
    c->field_valid = true;
    c->field_step = c->step;
    c->obs_step = -1;  // observables' terms formed on the previous field are stale
    return HPF_OK;
}

// Field of an arbitrary mesh D (tensor map tm when tm_ok) into the context's
// field buffer, clearing D_clear when given.  The tile must have been chosen
// (run_field ran before).  The context's mesh bookkeeping is not changed.
hpf_status field_from(hpf_ctx* c, const unsigned long long* D, const CUtensorMap& tm, bool tm_ok,
                      unsigned long long* D_clear, float4* G_out = nullptr) {
    float4* G = G_out ? G_out : c->G;
    if (!G_out) c->obs_step = -1;  // the context's field changes
    {
        StageScope sc(c, HPF_STAGE_FIELD, 1);
        if (c->S <= 4 && c->field_tile >= 0) {
            SingleFieldParams p;
            memset(&p, 0, sizeof p);
            p.R = 1;
            p.flag = c->dflag;
            fill_field_rep_mesh(c, c->field_tile, D, tm, tm_ok, D_clear, p.rep[0], p.blocks);
            p.rep[0].G = G;
            launch_field_tiled(p, c->S, c->field_tile, c->stream);
        } else {
            BatchFieldParams fp;
            memset(&fp, 0, sizeof fp);
            fp.R = 1;
            fp.coef = c->d_coef;
            fp.rep[0].g = c->geom;
            fp.rep[0].D = reinterpret_cast<const long long*>(D);
            fp.rep[0].G = G;
            fp.rep[0].D_clear = D_clear;
            fp.rep[0].blk_begin = 0;
            fp.blocks = (c->geom.gnodes + 255) / 256;
            launch_field_batch(fp, c->S, c->stream);
        }
    }
    LAUNCH_CHECK(c);
    return HPF_OK;
}

hpf_status refresh_field(hpf_ctx* c) {
    hpf_status s = scatter_current(c);
    if (s != HPF_OK) return s;
    return run_field(c);
}

// The field in force at the current step: refreshed when none is valid or the
// step is a refresh step that has not been done yet.
hpf_status ensure_field(hpf_ctx* c) {
    if (!c->field_valid || (c->step % c->p.field_every == 0 && c->field_step != c->step))
        return refresh_field(c);
    return HPF_OK;
}

// Reorder whole chains by the cell of their first bead (results do not depend on it).
hpf_status sort_beads(hpf_ctx* c) {
    {
        StageScope sc(c, HPF_STAGE_SORT, 0);
        SortBufs b = c->sb;
        if (!c->warp_mode) b.seg_start = nullptr;
        sc.kernels = launch_sort(b, c->st[c->cur], c->st[c->cur ^ 1], c->meta, c->meta2, c->n,
                                 c->C, c->geom, c->stream);
    }
    LAUNCH_CHECK(c);
    c->cur ^= 1;
    uint32_t* t = c->meta;
    c->meta = c->meta2;
    c->meta2 = t;
    int* u = c->sb.chain_of_in;
    c->sb.chain_of_in = c->sb.chain_of_out;
    c->sb.chain_of_out = u;
    c->last_sort_step = c->step;
    return HPF_OK;
}

// Launch `chunk` steps on the field in force; with fuse the last sub-step
// also scatters its positions into the other mesh (which must be zero).
// lerp_G2: a learned window in one launch (warp form, force_mode 0): the
// field (1 - j/K) G + (j/K) lerp_G2 at window step j, lerp_j0 at the first
// sub-step, lerp_inv_k = 1/K.
hpf_status advance(hpf_ctx* c, int chunk, bool fuse, const float4* lerp_G2 = nullptr,
                   int lerp_j0 = 0, float lerp_inv_k = 0.f, bool obs = false) {
    c->obs_step = -1;
    {
        StageScope sc(c, HPF_STAGE_STEP, c->n > 0 ? 1 : 0);
        if (c->warp_mode) {
            // the batch step kernel instantiated for one replica
            SingleStepParams p;
            memset(&p, 0, sizeof p);
            p.R = 1;
            p.n_sub = chunk;
            p.cur = c->cur;
            p.fuse = fuse ? 1 : 0;
            p.dnext = c->dmesh ^ 1;
            p.step0 = c->step;
            p.step_dev = nullptr;
            p.flag = c->dflag;
            BatchStepRep& q = p.rep[0];
            q.g = c->geom;
            q.c = c->sc;
            q.st[0] = c->st[0];
            q.st[1] = c->st[1];
            q.meta = c->meta;
            q.seg_start = c->sb.seg_start;
            q.seg_count = c->sb.seg_count;
            q.n_seg = c->sb.n_seg;
            q.G = c->G;
            q.D[0] = mesh_buf(c, 0);
            q.D[1] = mesh_buf(c, 1);
            if (lerp_G2)
                launch_step_warp_lerp(p, lerp_G2, lerp_j0, lerp_inv_k, c->C,
                                      step_thermostat(c->sc), c->stream);
            else if (obs)
                c->obs_nb = launch_step_warp_obs(p, c->C, step_thermostat(c->sc), c->obs_part,
                                                 (float)c->ec.half_dt_m, bond_ff(c->ec),
                                                 c->stream);
            else
                launch_step_warp_single(p, c->C, step_thermostat(c->sc), c->stream);
        } else
            launch_step(c->st[c->cur], c->st[c->cur ^ 1], c->meta, c->n, chunk, c->step, c->geom,
                        c->G, c->sc, fuse ? mesh_buf(c, c->dmesh ^ 1) : nullptr, c->dflag,
                        c->stream);
    }
    LAUNCH_CHECK(c);
    c->cur ^= 1;
    c->step += chunk;
    if (fuse) {
        c->dmesh ^= 1;
        c->mesh_step = c->step;
        c->next_zero = false;
    }
    if (obs && c->obs_nb > 0) c->obs_step = c->step;
    return HPF_OK;
}

// Nose-Hoover: `chunk` steps on the field in force (one launch per step plus
// one, see k_nh.cu); with fuse the last launch deposits its positions into
// the other mesh (which must be zero).
hpf_status advance_nh(hpf_ctx* c, int chunk, bool fuse) {
    c->obs_step = -1;
    {
        StageScope sc(c, HPF_STAGE_STEP, c->n > 0 ? chunk + 1 : 0);
        if (c->n > 0) {
            const size_t n = (size_t)c->n;
            NhParams p;
            memset(&p, 0, sizeof p);
            p.meta = c->meta;
            p.n = c->n;
            p.g = c->geom;
            p.G = c->G;
            p.c = c->sc;
            p.t = c->nhc;
            p.nh = c->nh;
            p.part = reinterpret_cast<float2*>(c->nh_part);  // one double's room per block
            p.flag = c->dflag;
            // one launch; the state and (after a force evaluation) the force buffers swap
            auto launch = [&](bool kick_drift, bool force_kick, unsigned long long* D_next) {
                p.in = c->st[c->cur];
                p.out = c->st[c->cur ^ 1];
                for (int a = 0; a < 3; ++a) {
                    p.Fin[a] = c->nh_F + ((size_t)c->nh_f * 3 + a) * n;
                    p.Fout[a] = c->nh_F + ((size_t)(c->nh_f ^ 1) * 3 + a) * n;
                }
                p.kick_drift = kick_drift ? 1 : 0;
                p.force_kick = force_kick ? 1 : 0;
                p.D_next = D_next;
                launch_nh_step(p, c->stream);
                c->cur ^= 1;
                if (force_kick) c->nh_f ^= 1;
            };
            // F_n and the thermostat at the first step (after a refresh or a call boundary)
            launch(false, true, nullptr);
            for (int j = 0; j < chunk; ++j) {
                const bool last = j == chunk - 1;
                launch(true, !last, (last && fuse) ? mesh_buf(c, c->dmesh ^ 1) : nullptr);
            }
        }
    }
    LAUNCH_CHECK(c);
    c->step += chunk;
    if (fuse) {
        c->dmesh ^= 1;
        c->mesh_step = c->step;
        c->next_zero = false;
    }
    return HPF_OK;
}

// The pending thermostat half step of the current step (the end of the last
// one) applied on the host to the on-step quantities of the state: returns
// the velocity scale and advances copies of xi, eta and K.
double nh_pending_half(const hpf_ctx* c, double& xi, double& eta, double& K) {
    const NhConsts& t = c->nhc;
    auto rate = [&](double k) { return t.dof_kT > 0.0 ? (2.0 * k / t.dof_kT - 1.0) * t.inv_tau2 : 0.0; };
    xi += 0.5 * t.h * rate(K);
    const double s = exp(-xi * t.h);
    K *= s * s;
    eta += xi * t.h;
    xi += 0.5 * t.h * rate(K);
    return s;
}

// The kernels' error word as copied to the host.
hpf_status flag_status(hpf_ctx* c, int word) {
    if (word & kFlagNonFinite)
        return fail(c, HPF_ERR_NONFINITE, "a position or velocity became non-finite");
    if (word & kFlagRange)
        return fail(c, HPF_ERR_OVERFLOW, "a bead left the +-2^18-cell coordinate range");
    if (word & kFlagTimeout) return fail(c, HPF_ERR_TIMEOUT, "a device wait timed out");
    return HPF_OK;
}

hpf_status check_flags(hpf_ctx* c) {
    CUDA_TRY(c, cudaMemcpyAsync(c->hflag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return flag_status(c, c->hflag[0]);
}

// The observables of the current step: kernels and the copies of the six
// sums (and the Nose-Hoover state) to the context's pinned mirrors, all
// asynchronous on the context's stream.
hpf_status energy_launch(hpf_ctx* c) {
    if (!c->has_state) return fail(c, HPF_ERR_STATE, "no state loaded");
    hpf_status s = ensure_field(c);
    if (s != HPF_OK) return s;
    // the mesh of the current positions for the field energy; when the last
    // hpf_step call ended here without depositing it, later calls deposit
    // their final positions in their last launch
    if (c->mesh_step != c->step && c->end_of_call_step == c->step) c->want_end_mesh = true;
    if ((s = scatter_current(c)) != HPF_OK) return s;
    {
        const long long* Dm = reinterpret_cast<const long long*>(mesh_buf(c, c->dmesh));
        if (c->obs_step == c->step) {
            // the bead terms came with the step launch: node sums and combination
            StageScope sc(c, HPF_STAGE_ENERGY, 2);
            launch_energy_nodes_only(c->n, c->geom, Dm, c->ec, c->obs_part, c->obs_nb,
                                     c->partials, c->d_out6, c->stream);
        } else {
            StageScope sc(c, HPF_STAGE_ENERGY, energy_launches(c->n, c->S));
            launch_energy(cur_state(c), c->meta, c->n, c->geom, c->G, c->sc, c->step, Dm, c->ec,
                          c->partials, c->d_out6, c->stream);
        }
    }
    LAUNCH_CHECK(c);
    CUDA_TRY(c, cudaMemcpyAsync(c->h_out6, c->d_out6, sizeof(double) * 6, cudaMemcpyDeviceToHost,
                                c->stream));
    if (c->nh)
        CUDA_TRY(c, cudaMemcpyAsync(c->h_nh, c->nh, sizeof(double) * 2, cudaMemcpyDeviceToHost,
                                    c->stream));
    // the error word as it stands after these kernels, for hpf_energy_finish
    CUDA_TRY(c, cudaMemcpyAsync(c->hflag + 7, c->dflag, sizeof(int), cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaEventRecord(c->energy_ev, c->stream));
    return HPF_OK;
}

// After the stream has reached energy_launch's copies: the six values.
void energy_finish(const hpf_ctx* c, double out[6]) {
    memcpy(out, c->h_out6, sizeof(double) * 6);
    if (c->nh) {
        // the kernels give the on-step velocity before the pending thermostat half step
        double xi = c->h_nh[0], eta = c->h_nh[1], K = out[0];
        const double sc = nh_pending_half(c, xi, eta, K);
        out[0] = K;
        out[3] = K + out[1] + out[2];
        out[4] *= sc;
        out[5] *= sc * sc;
    }
}

}  // namespace

extern "C" {

const char* hpf_status_string(hpf_status s) {
    switch (s) {
        case HPF_OK: return "ok";
        case HPF_ERR_INVALID: return "invalid argument";
        case HPF_ERR_CUDA: return "CUDA error";
        case HPF_ERR_NOMEM: return "out of device memory";
        case HPF_ERR_OVERFLOW: return "fixed-point or coordinate range exceeded";
        case HPF_ERR_NONFINITE: return "non-finite state";
        case HPF_ERR_TIMEOUT: return "device wait timed out";
        case HPF_ERR_STATE: return "no state loaded";
        case HPF_ERR_SCRATCH: return "mesh larger than the no-allocation scratch";
    }
    return "unknown status";
}

const char* hpf_last_error(const hpf_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

hpf_status hpf_init(const hpf_params* params, void* stream, hpf_ctx** out) {
    if (!out) return HPF_ERR_INVALID;
    *out = nullptr;
    const hpf_status v = validate_params(params);
    if (v != HPF_OK) return v;
    hpf_ctx* c = new hpf_ctx();
    c->p = *params;
    c->stream = (cudaStream_t)stream;
    c->n = params->n_beads;
    c->S = params->n_species;
    derive_constants(c);
    const size_t n = (size_t)(c->n > 0 ? c->n : 1);
    const size_t nodes = (size_t)c->geom.nodes;
    auto cleanup = [&](hpf_status s) {
        hpf_destroy(c);
        return s;
    };
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMalloc(&c->state_mem, sizeof(float) * 12 * n);
    e = e ? e : cudaMalloc(&c->meta, sizeof(uint32_t) * n);
    e = e ? e : cudaMalloc(&c->meta2, sizeof(uint32_t) * n);
    const long long K = sort_key_space(c->geom);
    const long long scan_words = scan_scratch_words(K > (long long)n ? K : (long long)n);
    const size_t sort_words = 13 * n + 2 * (n / 256 + 2) + 3 * (size_t)K + (size_t)scan_words + 64;
    e = e ? e : cudaMalloc(&c->sort_mem, sizeof(uint32_t) * sort_words);
    e = e ? e : cudaMalloc(&c->D, 2 * sizeof(unsigned long long) * nodes * c->S);
    e = e ? e : cudaMalloc(&c->G, sizeof(float4) * (size_t)c->geom.gnodes * c->S);
    e = e ? e : cudaMalloc(&c->field_stage, sizeof(float4) * nodes * c->S);
    e = e ? e : cudaMalloc(&c->d_coef, sizeof(FieldCoef));
    e = e ? e : cudaMalloc(&c->out_f, sizeof(float) * 6 * n);
    e = e ? e : cudaMalloc(&c->stage, stage_bytes((int)n));
    e = e ? e : cudaMalloc(&c->dflag, sizeof(int) * 8);
    e = e ? e : cudaMallocHost(&c->hflag, sizeof(int) * 8);
    e = e ? e : cudaMalloc(&c->partials,
                           sizeof(double) * energy_partials_needed(c->n, c->geom.nodes,
                                                                   c->p.n_species));
    e = e ? e : cudaMalloc(&c->d_out6, sizeof(double) * 8);
    e = e ? e : cudaMallocHost(&c->h_out6, sizeof(double) * 8);
    e = e ? e : cudaEventCreateWithFlags(&c->energy_ev, cudaEventDisableTiming);
    e = e ? e : cudaMalloc(&c->obs_part, sizeof(float2) * kBeadVals * step_warp_grid_cap());
    if (params->thermostat == 1) {
        e = e ? e : cudaMalloc(&c->nh, sizeof(NhDev));
        e = e ? e : cudaMalloc(&c->nh_part, sizeof(double) * (nh_blocks((int)n) + 1));
        e = e ? e : cudaMalloc(&c->nh_F, sizeof(float) * 6 * n);
        e = e ? e : cudaMallocHost(&c->h_nh, sizeof(double) * 2);
        e = e ? e : cudaMemsetAsync(c->nh, 0, sizeof(NhDev), c->stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cleanup(e == cudaErrorMemoryAllocation ? HPF_ERR_NOMEM : HPF_ERR_CUDA);
    }
    {
        uint32_t* w = (uint32_t*)c->sort_mem;
        SortBufs& b = c->sb;
        b.cstart = (int*)w; w += n;
        b.clen = (int*)w; w += n;
        b.tag0 = w; w += n;
        b.key = w; w += n;
        b.order_tmp = (int*)w; w += n;
        b.rank_of = (int*)w; w += n;
        b.newstart = w; w += n;
        b.chain_of_in = (int*)w; w += n;
        b.chain_of_out = (int*)w; w += n;
        b.seg_start = (int*)w; w += n;
        b.seg_count = (int*)w; w += n;
        b.seg_tmp = (int*)w; w += 2 * n;
        b.chunk_nseg = w; w += n / 256 + 2;
        b.chunk_off = w; w += n / 256 + 2;
        b.n_seg = (int*)w; w += 1;
        b.count = w; w += K;
        b.binoff = w; w += K;
        b.cursor = w; w += K;
        b.scratch = w;
    }
    for (int b = 0; b < 2; ++b) {
        float* base = c->state_mem + (size_t)b * 6 * n;
        c->st[b] = StateBuf{base, base + n, base + 2 * n, base + 3 * n, base + 4 * n, base + 5 * n};
    }
    if (cudaMemcpyAsync(c->d_coef, &c->coef, sizeof(FieldCoef), cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->dflag, 0, sizeof(int) * 8, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->D, 0, 2 * sizeof(unsigned long long) * nodes * c->S, c->stream) !=
            cudaSuccess)
        return cleanup(HPF_ERR_CUDA);
    c->next_zero = true;
    *out = c;
    return HPF_OK;
}

hpf_status hpf_destroy(hpf_ctx* c) {
    if (!c) return HPF_OK;
    cudaStreamSynchronize(c->stream);
    for (auto& e : c->ev_used) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    for (auto e : c->ev_free) cudaEventDestroy(e);
    cudaFree(c->state_mem);
    cudaFree(c->meta);
    cudaFree(c->meta2);
    cudaFree(c->sort_mem);
    cudaFree(c->D);
    cudaFree(c->G);
    cudaFree(c->field_stage);
    cudaFree(c->d_coef);
    cudaFree(c->out_f);
    cudaFree(c->stage);
    cudaFree(c->dflag);
    cudaFreeHost(c->hflag);
    cudaFree(c->partials);
    cudaFree(c->d_out6);
    cudaFreeHost(c->h_out6);
    if (c->energy_ev) cudaEventDestroy(c->energy_ev);
    cudaFree(c->obs_part);
    cudaFree(c->nh);
    cudaFree(c->nh_part);
    cudaFree(c->nh_F);
    cudaFreeHost(c->h_nh);
    if (c->up_stream) {
        cudaStreamSynchronize(c->up_stream);
        cudaStreamDestroy(c->up_stream);
    }
    for (int k = 0; k < 2; ++k) {
        if (c->up_done[k]) cudaEventDestroy(c->up_done[k]);
        if (c->up_free[k]) cudaEventDestroy(c->up_free[k]);
        cudaFree(c->up_stage[k]);
    }
    if (LearnedBufs* L = c->learned) {
        cudaFree(L->Dbase);
        cudaFree(L->Dp);
        cudaFree(L->x);
        cudaFree(L->dphi);
        cudaFree(L->snap);
        cudaFree(L->acc);
        cudaFreeHost(L->h_acc);
        cudaFree(L->G2);
        delete L;
    }
    cudaGetLastError();
    delete c;
    return HPF_OK;
}

hpf_status hpf_set_state(hpf_ctx* c, const float* pos, const float* vel, const int32_t* type,
                         const int32_t* bonds, int64_t n_bonds, int64_t step) {
    if (!c) return HPF_ERR_INVALID;
    const int n = c->n;
    if (step < 0) return fail(c, HPF_ERR_INVALID, "step must be >= 0");
    if (n > 0 && (!pos || !vel || !type))
        return fail(c, HPF_ERR_INVALID, "pos, vel and type are required");
    if (n_bonds < 0 || n_bonds >= (int64_t)(n > 0 ? n : 1) || (n_bonds > 0 && !bonds))
        return fail(c, HPF_ERR_INVALID, "n_bonds must be in [0, n_beads) with a bond array");
    char* stg = (char*)c->stage;
    float* spos = (float*)stg;
    float* svel = spos + 3 * (size_t)n;
    int32_t* stype = (int32_t*)(svel + 3 * (size_t)n);
    int32_t* sbond = stype + n;
    if (n > 0) {
        CUDA_TRY(c, cudaMemcpyAsync(spos, pos, sizeof(float) * 3 * n, cudaMemcpyDefault, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(svel, vel, sizeof(float) * 3 * n, cudaMemcpyDefault, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(stype, type, sizeof(int32_t) * n, cudaMemcpyDefault, c->stream));
    }
    if (n_bonds > 0)
        CUDA_TRY(c, cudaMemcpyAsync(sbond, bonds, sizeof(int32_t) * 2 * n_bonds, cudaMemcpyDefault,
                                    c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->dflag, 0, sizeof(int) * 8, c->stream));
    c->cur = 0;
    {
        StageScope sc(c, HPF_STAGE_OTHER, (n > 0) + (n_bonds > 0));
        launch_stage_state(spos, svel, stype, n, c->S, c->st[0], c->meta, c->dflag + 1,
                           c->stream);
        launch_mark_bonds(sbond, n_bonds, n, c->meta, c->dflag + 1, c->stream);
    }
    {
        StageScope sc(c, HPF_STAGE_SORT, 0);
        sc.kernels = launch_chain_build_heads(c->meta, n, c->sb.newstart, c->sb.scratch, c->stream);
    }
    LAUNCH_CHECK(c);
    CUDA_TRY(c, cudaMemcpyAsync(c->hflag, c->dflag, sizeof(int) * 8, cudaMemcpyDeviceToHost,
                                c->stream));
    if (n > 0) {
        CUDA_TRY(c, cudaMemcpyAsync(c->hflag + 5, c->sb.newstart + (n - 1), sizeof(uint32_t),
                                    cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(c->hflag + 6, c->meta + (n - 1), sizeof(uint32_t),
                                    cudaMemcpyDeviceToHost, c->stream));
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->has_state = false;
    c->field_valid = false;
    if (c->hflag[1]) return fail(c, HPF_ERR_INVALID, "%d bead species out of range", c->hflag[1]);
    if (c->hflag[2]) return fail(c, HPF_ERR_NONFINITE, "%d beads with non-finite state", c->hflag[2]);
    if (c->hflag[3])
        return fail(c, HPF_ERR_INVALID, "%d bonds do not join consecutive tags (i, i+1)",
                    c->hflag[3]);
    if (c->hflag[4]) return fail(c, HPF_ERR_INVALID, "%d bonds given twice", c->hflag[4]);
    c->C = 0;
    if (n > 0) {
        const uint32_t last_meta = (uint32_t)c->hflag[6];
        c->C = c->hflag[5] + ((last_meta & kBondPrev) ? 0 : 1);
        {
            StageScope sc(c, HPF_STAGE_SORT, 2);
            CUDA_TRY(c, cudaMemsetAsync(c->dflag + 7, 0, sizeof(int), c->stream));
            launch_chain_build(c->meta, c->sb.newstart, n, c->C, c->sb.cstart, c->sb.tag0,
                               c->sb.chain_of_in, c->sb.clen, c->dflag + 7, c->stream);
        }
        LAUNCH_CHECK(c);
        CUDA_TRY(c, cudaMemcpyAsync(c->hflag + 7, c->dflag + 7, sizeof(int),
                                    cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        c->max_chain = c->hflag[7];
    }
    c->warp_mode = n > 0 && c->max_chain <= 64;
    c->step = step;
    c->mesh_step = -1;
    c->part_step = -1;
    hpf_status s2 = sort_beads(c);
    if (s2 != HPF_OK) return s2;
    c->step = step;
    c->field_step = -1;
    c->obs_step = -1;
    if (c->nh) {
        // a loaded state starts with the thermostat at rest (hpf_set_thermostat restores one)
        CUDA_TRY(c, cudaMemsetAsync(c->nh, 0, sizeof(NhDev), c->stream));
    }
    c->has_state = true;
    return HPF_OK;
}

// New state (tag order, device staging) into storage order, its density
// deposited into the other mesh in the same pass: that mesh becomes the
// context's, holding the density of the positions at `step`.
static hpf_status repermute_deposit(hpf_ctx* c, const float* pos_tag, const float* vel_tag,
                                    long long step) {
    unsigned long long* dst = mesh_buf(c, c->dmesh ^ 1);
    if (!c->next_zero)
        CUDA_TRY(c, cudaMemsetAsync(dst, 0, sizeof(unsigned long long) * mesh_words(c), c->stream));
    {
        StageScope sc(c, HPF_STAGE_OTHER, 1);
        launch_repermute(pos_tag, vel_tag, c->meta, c->n, cur_state(c), c->geom, dst, c->dflag,
                         c->stream);
    }
    LAUNCH_CHECK(c);
    c->dmesh ^= 1;
    c->next_zero = false;
    c->step = step;
    c->mesh_step = step;
    c->end_mesh_unused = false;
    c->obs_step = -1;
    return HPF_OK;
}

hpf_status hpf_update_state(hpf_ctx* c, const float* pos, const float* vel, int64_t step) {
    if (!c) return HPF_ERR_INVALID;
    if (!c->has_state) return fail(c, HPF_ERR_STATE, "no state loaded");
    if (step < 0) return fail(c, HPF_ERR_INVALID, "step must be >= 0");
    const int n = c->n;
    if (n == 0) {
        c->step = step;
        c->field_valid = false;
        c->mesh_step = -1;
        c->part_step = -1;
        return HPF_OK;
    }
    if (!pos || !vel) return fail(c, HPF_ERR_INVALID, "pos and vel are required");
    float* spos = (float*)c->stage;
    float* svel = spos + 3 * (size_t)n;
    CUDA_TRY(c, cudaMemcpyAsync(spos, pos, sizeof(float) * 3 * n, cudaMemcpyDefault, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(svel, vel, sizeof(float) * 3 * n, cudaMemcpyDefault, c->stream));
    hpf_status s = repermute_deposit(c, spos, svel, step);
    if (s != HPF_OK) return s;
    c->field_valid = false;
    c->part_step = -1;
    return HPF_OK;
}

// The copy stream, events and staging slots of pipelined uploads, made on
// first use.  up_ready is set only once all of them exist; a failure part way
// releases what was made, so a later call starts over.
static hpf_status upload_setup(hpf_ctx* c) {
    cudaError_t e = cudaStreamCreateWithFlags(&c->up_stream, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&c->up_done[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->up_free[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&c->up_stage[k], sizeof(float) * 6 * (size_t)c->n);
    }
    if (e == cudaSuccess) {
        c->up_ready = true;
        return HPF_OK;
    }
    cudaGetLastError();
    for (int k = 0; k < 2; ++k) {
        if (c->up_done[k]) cudaEventDestroy(c->up_done[k]);
        if (c->up_free[k]) cudaEventDestroy(c->up_free[k]);
        cudaFree(c->up_stage[k]);
        c->up_done[k] = c->up_free[k] = nullptr;
        c->up_stage[k] = nullptr;
    }
    if (c->up_stream) cudaStreamDestroy(c->up_stream);
    c->up_stream = nullptr;
    return fail(c, e == cudaErrorMemoryAllocation ? HPF_ERR_NOMEM : HPF_ERR_CUDA,
                "upload set-up: %s", cudaGetErrorString(e));
}

hpf_status hpf_upload_state(hpf_ctx* c, const float* pos, const float* vel) {
    if (!c) return HPF_ERR_INVALID;
    if (!c->has_state) return fail(c, HPF_ERR_STATE, "no state loaded");
    if (c->up_pending) return fail(c, HPF_ERR_STATE, "an upload is pending (hpf_apply_state first)");
    const int n = c->n;
    if (n > 0) {
        if (!pos || !vel) return fail(c, HPF_ERR_INVALID, "pos and vel are required");
        if (!c->up_ready) {
            const hpf_status s = upload_setup(c);
            if (s != HPF_OK) return s;
        }
        const int k = c->up_slot;
        float* spos = c->up_stage[k];
        float* svel = spos + 3 * (size_t)n;
        // the slot is free once the permutation that last read it has run
        CUDA_TRY(c, cudaStreamWaitEvent(c->up_stream, c->up_free[k], 0));
        CUDA_TRY(c, cudaMemcpyAsync(spos, pos, sizeof(float) * 3 * n, cudaMemcpyDefault,
                                    c->up_stream));
        CUDA_TRY(c, cudaMemcpyAsync(svel, vel, sizeof(float) * 3 * n, cudaMemcpyDefault,
                                    c->up_stream));
        CUDA_TRY(c, cudaEventRecord(c->up_done[k], c->up_stream));
    }
    c->up_pending = true;
    return HPF_OK;
}

hpf_status hpf_apply_state(hpf_ctx* c, int64_t step) {
    if (!c) return HPF_ERR_INVALID;
    if (!c->has_state) return fail(c, HPF_ERR_STATE, "no state loaded");
    if (!c->up_pending) return fail(c, HPF_ERR_STATE, "no upload pending (hpf_upload_state first)");
    if (step < 0) return fail(c, HPF_ERR_INVALID, "step must be >= 0");
    const int n = c->n;
    if (n > 0) {
        const int k = c->up_slot;
        CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->up_done[k], 0));
        hpf_status s = repermute_deposit(c, c->up_stage[k], c->up_stage[k] + 3 * (size_t)n, step);
        if (s != HPF_OK) return s;
        CUDA_TRY(c, cudaEventRecord(c->up_free[k], c->stream));
        c->up_slot ^= 1;
    } else {
        c->mesh_step = -1;
    }
    c->up_pending = false;
    c->step = step;
    c->field_valid = false;
    c->part_step = -1;
    return HPF_OK;
}

hpf_status hpf_get_state(hpf_ctx* c, float* pos, float* vel, int64_t* step) {
    if (!c) return HPF_ERR_INVALID;
    if (!c->has_state) return fail(c, HPF_ERR_STATE, "no state loaded");
    float* pt = c->out_f;
    float* vt = c->out_f + 3 * (size_t)c->n;
    {
        StageScope sc(c, HPF_STAGE_OTHER, c->n > 0 ? 1 : 0);
        launch_unpermute(cur_state(c), c->meta, c->n, pt, vt, c->dflag, c->stream);
    }
    LAUNCH_CHECK(c);
    hpf_status s;
    if ((s = copy_out(c, pos, pt, sizeof(float) * 3 * c->n)) != HPF_OK) return s;
    if ((s = copy_out(c, vel, vt, sizeof(float) * 3 * c->n)) != HPF_OK) return s;
    if (step) *step = c->step;
    return check_flags(c);
}

hpf_status hpf_get_order(hpf_ctx* c, int32_t* order) {
    if (!c) return HPF_ERR_INVALID;
    if (c->n > 0 && !order) return fail(c, HPF_ERR_INVALID, "order is required");
    if (!c->has_state) return fail(c, HPF_ERR_STATE, "no state loaded");
    {
        StageScope sc(c, HPF_STAGE_OTHER, c->n > 0 ? 1 : 0);
        launch_order(c->meta, c->n, (int32_t*)c->out_f, c->stream);
    }
    LAUNCH_CHECK(c);
    return copy_out(c, order, c->out_f, sizeof(int32_t) * c->n);
}

hpf_status hpf_scatter_density(hpf_ctx* c, int64_t* D_out) {
    if (!c) return HPF_ERR_INVALID;
    if (!c->has_state) return fail(c, HPF_ERR_STATE, "no state loaded");
    hpf_status s = scatter_current(c);
    if (s != HPF_OK) return s;
    return copy_out(c, D_out, mesh_buf(c, c->dmesh), sizeof(unsigned long long) * mesh_words(c));
}

hpf_status hpf_field(hpf_ctx* c, const int64_t* D_in, float* field_out) {
    if (!c) return HPF_ERR_INVALID;
    if (!c->has_state) return fail(c, HPF_ERR_STATE, "no state loaded");
    if (D_in) {
        CUDA_TRY(c, cudaMemcpyAsync(mesh_buf(c, c->dmesh ^ 1), D_in,
                                    sizeof(long long) * mesh_words(c), cudaMemcpyDefault,
                                    c->stream));
        c->dmesh ^= 1;
        c->mesh_step = -1;  // an injected mesh is not the density of the positions
        c->part_step = -1;
        c->next_zero = false;
    }
    hpf_status s = run_field(c);
    if (s != HPF_OK) return s;
    if (!field_out) return HPF_OK;
    {
        StageScope sc(c, HPF_STAGE_OTHER, 1);
        launch_unpad_field(c->G, c->geom, c->S, c->field_stage, c->stream);
    }
    LAUNCH_CHECK(c);
    return copy_out(c, field_out, c->field_stage, sizeof(float4) * mesh_words(c));
}

hpf_status hpf_forces(hpf_ctx* c, float* F_out, int32_t which) {
    if (!c) return HPF_ERR_INVALID;
    if (which < 1 || which > 3) return fail(c, HPF_ERR_INVALID, "which must be 1, 2 or 3");
    if (c->n > 0 && !F_out) return fail(c, HPF_ERR_INVALID, "F_out is required");
    if (!c->has_state) return fail(c, HPF_ERR_STATE, "no state loaded");
    hpf_status s;
    if ((which & HPF_FORCE_FIELD) && (s = ensure_field(c)) != HPF_OK) return s;
    {
        StageScope sc(c, HPF_STAGE_OTHER, c->n > 0 ? 1 : 0);
        launch_forces(cur_state(c), c->meta, c->n, c->geom, c->G, c->sc, which, c->out_f,
                      c->stream);
    }
    LAUNCH_CHECK(c);
    return copy_out(c, F_out, c->out_f, sizeof(float) * 3 * c->n);
}

// Whether the launch of `chunk` steps from the current step deposits its final
// positions into the other mesh: always when it ends on a refresh step and
// that mesh is already clear (the field kernel clears it); also, as the last
// launch of an hpf_step call, when calls have been followed by the
// observables of their final state (the other mesh is cleared first if
// need be: a memset costs far less than the scatter it saves).
// Such a launch, when it does not end on a refresh step (where F_n needs the
// new field), also forms the observables' bead terms of its final state
// (obs) if the step kernel supports them here: warp form, Langevin or no
// thermostat, bonds only, interpolated-gradient force.
static hpf_status plan_deposit(hpf_ctx* c, long long chunk, bool last, bool& fuse, bool& obs) {
    const bool refresh_end = (c->step + chunk) % c->p.field_every == 0;
    fuse = refresh_end && c->next_zero;
    obs = false;
    if (!fuse && last && c->want_end_mesh && c->n > 0) {
        if (!c->next_zero) {
            CUDA_TRY(c, cudaMemsetAsync(mesh_buf(c, c->dmesh ^ 1), 0,
                                        sizeof(unsigned long long) * mesh_words(c), c->stream));
            c->next_zero = true;
        }
        fuse = true;
    }
    if (fuse && last && !refresh_end) {
        c->end_mesh_unused = true;
        obs = c->warp_mode && !c->nh && step_thermostat(c->sc) <= 1 && c->sc.force_mode == 0 &&
              bonded_level(c->sc) == 0;
    }
    return HPF_OK;
}

hpf_status hpf_step(hpf_ctx* c, int32_t n_steps) {
    if (!c) return HPF_ERR_INVALID;
    if (n_steps < 0) return fail(c, HPF_ERR_INVALID, "n_steps must be >= 0");
    if (!c->has_state) return fail(c, HPF_ERR_STATE, "no state loaded");
    const long long fe = c->p.field_every;
    long long left = n_steps;
    if (n_steps > 0) {
        // an end deposit nobody read: stop making them
        if (c->end_mesh_unused) c->want_end_mesh = false;
        c->end_mesh_unused = false;
    }
    if (c->nh) {
        while (left > 0) {
            hpf_status s = ensure_field(c);
            if (s != HPF_OK) return s;
            long long chunk = fe - (c->step % fe);
            if (chunk > left) chunk = left;
            if (c->p.sort_every > 0 && c->step - c->last_sort_step >= c->p.sort_every) {
                if ((s = sort_beads(c)) != HPF_OK) return s;
            }
            bool fuse, obs;
            if ((s = plan_deposit(c, chunk, chunk == left, fuse, obs)) != HPF_OK) return s;
            if ((s = advance_nh(c, (int)chunk, fuse)) != HPF_OK) return s;
            left -= chunk;
        }
        c->end_of_call_step = c->step;
        return HPF_OK;
    }
    while (left > 0) {
        hpf_status s = ensure_field(c);
        if (s != HPF_OK) return s;
        long long chunk = fe - (c->step % fe);  // steps until the next refresh
        if (chunk > left) chunk = left;
        // the halo form recomputes `chunk` beads per side; the warp form has no halo
        if (chunk > (c->warp_mode ? 64 : step_halo_max()))
            chunk = c->warp_mode ? 64 : step_halo_max();
        if (c->p.sort_every > 0 && c->step - c->last_sort_step >= c->p.sort_every) {
            if ((s = sort_beads(c)) != HPF_OK) return s;
        }
        bool fuse, obs;
        if ((s = plan_deposit(c, chunk, chunk == left, fuse, obs)) != HPF_OK) return s;
        if ((s = advance(c, (int)chunk, fuse, nullptr, 0, 0.f, obs)) != HPF_OK) return s;
        left -= chunk;
    }
    c->end_of_call_step = c->step;
    return HPF_OK;
}

hpf_status hpf_set_tag_base(hpf_ctx* c, int64_t tag_base) {
    if (!c) return HPF_ERR_INVALID;
    if (tag_base < 0 || tag_base + (int64_t)c->n > (int64_t)HPF_MAX_BEADS + 1)
        return fail(c, HPF_ERR_INVALID, "tag_base + n_beads must stay within 2^24");
    c->sc.tag_base = (uint32_t)tag_base;
    c->obs_step = -1;  // the noise of F_n depends on it
    return HPF_OK;
}

// hpf_step that stops where a refresh is due: the first call there hands out
// the part's own density of the current positions (deposited by the last
// launch, or scattered now) for the caller to sum over all parts; the next
// call takes the mesh as it then stands for the field.
hpf_status hpf_step_partial(hpf_ctx* c, int32_t n_steps, int32_t* steps_done, int64_t** mesh) {
    if (!c) return HPF_ERR_INVALID;
    if (!steps_done || !mesh) return fail(c, HPF_ERR_INVALID, "steps_done and mesh are required");
    *steps_done = 0;
    *mesh = nullptr;
    if (n_steps < 0) return fail(c, HPF_ERR_INVALID, "n_steps must be >= 0");
    if (!c->has_state) return fail(c, HPF_ERR_STATE, "no state loaded");
    if (c->nh)
        return fail(c, HPF_ERR_INVALID, "Nose-Hoover couples every bead each step: no partial steps");
    const long long fe = c->p.field_every;
    long long left = n_steps;
    for (;;) {
        hpf_status s;
        const bool due = !c->field_valid || (c->step % fe == 0 && c->field_step != c->step);
        if (due) {
            if (c->part_step != c->step) {
                if ((s = scatter_current(c)) != HPF_OK) return s;
                c->part_step = c->step;
                *mesh = reinterpret_cast<int64_t*>(mesh_buf(c, c->dmesh));
                return HPF_OK;
            }
            // the mesh holds the sum over the parts now, not this part's density
            if ((s = run_field(c)) != HPF_OK) return s;
            c->mesh_step = -1;
        }
        if (left == 0) return HPF_OK;
        long long chunk = fe - (c->step % fe);
        if (chunk > left) chunk = left;
        if (chunk > (c->warp_mode ? 64 : step_halo_max()))
            chunk = c->warp_mode ? 64 : step_halo_max();
        if (c->p.sort_every > 0 && c->step - c->last_sort_step >= c->p.sort_every) {
            if ((s = sort_beads(c)) != HPF_OK) return s;
        }
        const bool fuse = ((c->step + chunk) % fe == 0) && c->next_zero;
        if ((s = advance(c, (int)chunk, fuse)) != HPF_OK) return s;
        left -= chunk;
        *steps_done += (int32_t)chunk;
    }
}

hpf_status hpf_energy(hpf_ctx* c, double out[6]) {
    if (!c || !out) return fail(c, HPF_ERR_INVALID, "out is required");
    if (c->energy_pending) return fail(c, HPF_ERR_STATE, "hpf_energy_start is pending");
    hpf_status s = energy_launch(c);
    if (s != HPF_OK) return s;
    if ((s = check_flags(c)) != HPF_OK) return s;
    energy_finish(c, out);
    return HPF_OK;
}

hpf_status hpf_energy_start(hpf_ctx* c) {
    if (!c) return HPF_ERR_INVALID;
    if (c->energy_pending) return fail(c, HPF_ERR_STATE, "hpf_energy_start is pending");
    const hpf_status s = energy_launch(c);
    if (s != HPF_OK) return s;
    c->energy_pending = true;
    return HPF_OK;
}

hpf_status hpf_energy_finish(hpf_ctx* c, double out[6]) {
    if (!c || !out) return fail(c, HPF_ERR_INVALID, "out is required");
    if (!c->energy_pending) return fail(c, HPF_ERR_STATE, "no hpf_energy_start pending");
    c->energy_pending = false;
    // waits for the observables' own copies only: work enqueued after
    // hpf_energy_start (the next step's upload, permutation, step) keeps running
    CUDA_TRY(c, cudaEventSynchronize(c->energy_ev));
    const hpf_status s = flag_status(c, c->hflag[7]);
    if (s != HPF_OK) return s;
    energy_finish(c, out);
    return HPF_OK;
}

hpf_status hpf_get_thermostat(hpf_ctx* c, double out[2]) {
    if (!c || !out) return fail(c, HPF_ERR_INVALID, "out is required");
    if (!c->nh) return fail(c, HPF_ERR_INVALID, "the context has no Nose-Hoover thermostat");
    // hpf_energy_finish reads the pinned mirror the copy below would overwrite
    if (c->energy_pending) return fail(c, HPF_ERR_STATE, "hpf_energy_start is pending");
    CUDA_TRY(c, cudaMemcpyAsync(c->h_nh, c->nh, sizeof(double) * 2, cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    out[0] = c->h_nh[0];
    out[1] = c->h_nh[1];
    return HPF_OK;
}

hpf_status hpf_set_thermostat(hpf_ctx* c, const double in[2]) {
    if (!c || !in) return fail(c, HPF_ERR_INVALID, "in is required");
    if (!c->nh) return fail(c, HPF_ERR_INVALID, "the context has no Nose-Hoover thermostat");
    if (!isfinite(in[0]) || !isfinite(in[1])) return fail(c, HPF_ERR_INVALID, "non-finite xi or eta");
    if (c->energy_pending) return fail(c, HPF_ERR_STATE, "hpf_energy_start is pending");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // the pinned mirror may still be in use
    c->h_nh[0] = in[0];
    c->h_nh[1] = in[1];
    CUDA_TRY(c, cudaMemcpyAsync(c->nh, c->h_nh, sizeof(double) * 2, cudaMemcpyHostToDevice,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return HPF_OK;
}

hpf_status hpf_nh_conserved(hpf_ctx* c, double* H) {
    if (!c || !H) return fail(c, HPF_ERR_INVALID, "H is required");
    if (!c->nh) return fail(c, HPF_ERR_INVALID, "the context has no Nose-Hoover thermostat");
    double e[6];
    hpf_status s = hpf_energy(c, e);
    if (s != HPF_OK) return s;
    // hpf_energy left the state's xi, eta in the pinned mirror and the kinetic
    // energy before the pending half step in the energy mirror
    double xi = c->h_nh[0], eta = c->h_nh[1], K = c->h_out6[0];
    nh_pending_half(c, xi, eta, K);
    *H = e[3] + c->nhc.dof_kT * (0.5 * c->p.nh_tau * c->p.nh_tau * xi * xi + eta);
    return HPF_OK;
}

hpf_status hpf_selftest_timeout(hpf_ctx* c, double* seconds) {
    if (!c) return HPF_ERR_INVALID;
    CUDA_TRY(c, cudaMemcpyAsync(c->hflag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const int before = c->hflag[0];
    const auto t0 = std::chrono::steady_clock::now();
    launch_wait_selftest(c->dflag, c->stream);
    LAUNCH_CHECK(c);
    CUDA_TRY(c, cudaMemcpyAsync(c->hflag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const auto t1 = std::chrono::steady_clock::now();
    const int after = c->hflag[0];
    // the flag word as it was: the self-test is its only writer meanwhile
    c->hflag[0] = before;
    CUDA_TRY(c, cudaMemcpyAsync(c->dflag, c->hflag, sizeof(int), cudaMemcpyHostToDevice,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (seconds) *seconds = std::chrono::duration<double>(t1 - t0).count();
    return (after & kFlagTimeout) ? HPF_ERR_TIMEOUT : HPF_OK;
}

hpf_status hpf_field_tile(const hpf_ctx* c, int32_t shape[3], int32_t* uses_tma) {
    if (!c) return HPF_ERR_INVALID;
    int t[3] = {0, 0, 0};
    if (c->field_tile >= 0) field_tile_shape(c->field_tile, t);
    if (shape)
        for (int a = 0; a < 3; ++a) shape[a] = t[a];
    if (uses_tma) *uses_tma = (c->field_tile >= 0 && c->tmap_ok) ? 1 : 0;
    return HPF_OK;
}

hpf_status hpf_set_field_tile(hpf_ctx* c, int32_t tile) {
    if (!c || tile < -1 || tile >= field_tile_candidates()) return HPF_ERR_INVALID;
    c->field_tile = tile;
    return HPF_OK;
}

hpf_status hpf_profile(hpf_ctx* c, int32_t enable) {
    if (!c) return HPF_ERR_INVALID;
    c->profiling = enable != 0;
    return HPF_OK;
}

hpf_status hpf_profile_read(hpf_ctx* c, double ms[HPF_STAGE_COUNT],
                            int64_t launches[HPF_STAGE_COUNT]) {
    if (!c) return HPF_ERR_INVALID;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    double acc[HPF_STAGE_COUNT] = {};
    for (auto& e : c->ev_used) {
        float t = 0.f;
        CUDA_TRY(c, cudaEventElapsedTime(&t, e.a, e.b));
        acc[e.stage] += t;
        c->ev_free.push_back(e.a);
        c->ev_free.push_back(e.b);
    }
    c->ev_used.clear();
    for (int k = 0; k < HPF_STAGE_COUNT; ++k) {
        if (ms) ms[k] = acc[k];
        if (launches) launches[k] = c->launches[k];
        c->launches[k] = 0;
    }
    return HPF_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches

struct hpf_batch {
    int R = 0;
    cudaStream_t stream = nullptr;
    std::vector<hpf_ctx*> rep;
    bool use_graphs = true;
    FieldCoef* d_coef = nullptr;  // [R]
    long long* d_step = nullptr;  // step counter read by graph replays
    cudaGraphExec_t gexec = nullptr;
    std::vector<const void*> graph_key;  // buffers the captured graph refers to
    std::vector<int> rep_tile;           // stencil tile shape chosen per replica mesh (empty: not yet)
    std::string err;
};

namespace {

hpf_status bfail(hpf_batch* b, hpf_status s, const char* msg) {
    if (b) b->err = msg;
    return s;
}

// The batched stencil over all replicas, each reading its mesh buffer
// dmesh ^ flip: one tiled launch per distinct tile shape among the replicas
// (each replica keeps the shape the autotuner picked for its mesh).
void launch_batch_fields(hpf_batch* b, int flip) {
    const int S = b->rep[0]->S;
    std::vector<int> shapes;
    for (int t : b->rep_tile)
        if (std::find(shapes.begin(), shapes.end(), t) == shapes.end()) shapes.push_back(t);
    for (int t : shapes) {
        TiledFieldParams p;
        memset(&p, 0, sizeof p);
        p.flag = b->rep[0]->dflag;
        for (int r = 0; r < b->R; ++r) {
            if (b->rep_tile[r] != t) continue;
            hpf_ctx* c = b->rep[r];
            fill_field_rep(c, t, c->dmesh ^ flip, p.rep[p.R++], p.blocks);
        }
        launch_field_tiled(p, S, t, b->stream);
    }
}

// Tile shapes: every candidate timed on each replica's own mesh gives a shape
// per replica; the grouped launches this needs (one per distinct shape) are
// then timed against the best single shape for all replicas in one launch,
// and the faster of the two is kept.
void batch_autotune(hpf_batch* b) {
    const int S = b->rep[0]->S;
    std::vector<int> per(b->R, 0);
    for (int r = 0; r < b->R; ++r) {
        hpf_ctx* c = b->rep[r];
        per[r] = autotune_tile<TiledFieldParams>(b->stream, S, [&](int t, TiledFieldParams& p) {
            memset(&p, 0, sizeof p);
            p.flag = c->dflag;
            p.R = 1;
            fill_field_rep(c, t, c->dmesh, p.rep[0], p.blocks);
        });
    }
    const int uni = autotune_tile<TiledFieldParams>(b->stream, S, [&](int t, TiledFieldParams& p) {
        memset(&p, 0, sizeof p);
        p.flag = b->rep[0]->dflag;
        for (int r = 0; r < b->R; ++r) {
            hpf_ctx* c = b->rep[r];
            fill_field_rep(c, t, c->dmesh, p.rep[p.R++], p.blocks);
        }
    });
    cudaEvent_t e0, e1;
    float ms[2] = {0.f, 0.f};
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        for (int k = 0; k < 2; ++k) {
            b->rep_tile = k == 0 ? per : std::vector<int>(b->R, uni);
            launch_batch_fields(b, 0);  // warm
            cudaEventRecord(e0, b->stream);
            for (int rep = 0; rep < 3; ++rep) launch_batch_fields(b, 0);
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms[k], e0, e1) != cudaSuccess)
                ms[k] = 0.f;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    cudaGetLastError();
    b->rep_tile = (ms[0] > 0.f && ms[0] < ms[1]) ? per : std::vector<int>(b->R, uni);
}

// Batched refresh of the replicas whose field is due (all of them in steady state).
hpf_status batch_refresh(hpf_batch* b) {
    hpf_ctx* c0 = b->rep[0];
    int due_n = 0;
    for (int r = 0; r < b->R; ++r) {
        hpf_ctx* c = b->rep[r];
        const bool due = !c->field_valid || (c->step % c->p.field_every == 0 && c->field_step != c->step);
        if (!due) continue;
        hpf_status s = scatter_current(c);
        if (s != HPF_OK) return s;
        ++due_n;
    }
    if (due_n == 0) return HPF_OK;
    if (due_n != b->R || c0->S > 4) {
        // only some replicas are due (or no tiled stencil): refresh them one by one
        for (int r = 0; r < b->R; ++r) {
            hpf_ctx* c = b->rep[r];
            const bool due = !c->field_valid || (c->step % c->p.field_every == 0 && c->field_step != c->step);
            if (due) {
                hpf_status s = run_field(c);
                if (s != HPF_OK) return s;
            }
        }
        return HPF_OK;
    }
    if (b->rep_tile.empty()) batch_autotune(b);
    {
        StageScope sc(c0, HPF_STAGE_FIELD, 1);
        launch_batch_fields(b, 0);
    }
    LAUNCH_CHECK(c0);
    for (auto* c : b->rep) {
        c->next_zero = true;
        c->field_valid = true;
        c->field_step = c->step;
        c->obs_step = -1;
    }
    return HPF_OK;
}

void fill_step_params(hpf_batch* b, BatchStepParams& p, int n_sub, bool fuse) {
    memset(&p, 0, sizeof p);
    hpf_ctx* c0 = b->rep[0];
    p.R = b->R;
    p.n_sub = n_sub;
    p.cur = c0->cur;
    p.fuse = fuse ? 1 : 0;
    p.dnext = c0->dmesh ^ 1;
    p.step0 = c0->step;
    p.step_dev = nullptr;
    p.flag = c0->dflag;
    for (int r = 0; r < b->R; ++r) {
        hpf_ctx* c = b->rep[r];
        BatchStepRep& q = p.rep[r];
        q.g = c->geom;
        q.c = c->sc;
        q.st[0] = c->st[0];
        q.st[1] = c->st[1];
        q.meta = c->meta;
        q.seg_start = c->sb.seg_start;
        q.seg_count = c->sb.seg_count;
        q.n_seg = c->sb.n_seg;
        q.G = c->G;
        q.D[0] = mesh_buf(c, 0);
        q.D[1] = mesh_buf(c, 1);
    }
}

int batch_max_segments(hpf_batch* b) {
    int m = 0;
    for (auto* c : b->rep) m += c->C;
    return m;
}

// The step kernels' thermostat for all replicas (they share the thermostat
// kind; a replica without friction or collisions adds zero noise or never
// collides under the kind's instantiation).
int batch_thermostat(hpf_batch* b) {
    int t = 0;
    for (auto* c : b->rep) t = std::max(t, step_thermostat(c->sc));
    return t;
}

void batch_advance(hpf_batch* b, long long chunk, bool fuse) {
    for (auto* c : b->rep) {
        c->obs_step = -1;
        c->cur ^= 1;
        c->step += chunk;
        if (fuse) {
            c->dmesh ^= 1;
            c->mesh_step = c->step;
            c->next_zero = false;
        }
    }
}

std::vector<const void*> batch_key(hpf_batch* b) {
    std::vector<const void*> k;
    for (auto* c : b->rep) {
        k.push_back(c->meta);
        k.push_back((const void*)(intptr_t)(c->cur * 2 + c->dmesh));
    }
    return k;
}

// Capture two steady-state field periods (refresh + fused step, twice), after
// which every buffer parity is back where it started, so the graph can be
// replayed; the step number comes from b->d_step, advanced inside the graph.
hpf_status batch_capture(hpf_batch* b) {
    hpf_ctx* c0 = b->rep[0];
    const int fe = c0->p.field_every;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    CUDA_TRY(c0, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    for (int half = 0; half < 2; ++half) {
        launch_batch_fields(b, half);
        BatchStepParams sp;
        fill_step_params(b, sp, fe, true);
        sp.cur = c0->cur ^ half;
        sp.dnext = c0->dmesh ^ half ^ 1;
        sp.step_dev = b->d_step;
        launch_step_warp_batch(sp, batch_max_segments(b), batch_thermostat(b), b->stream);
        launch_advance_counter(b->d_step, fe, b->stream);
    }
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c0, HPF_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b->gexec = nullptr;
        return fail(c0, HPF_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    b->graph_key = batch_key(b);
    return HPF_OK;
}

}  // namespace

extern "C" {

hpf_status hpf_batch_init(const hpf_params* params, int32_t n_replicas, void* stream,
                          hpf_batch** out) {
    if (!out) return HPF_ERR_INVALID;
    *out = nullptr;
    if (!params || n_replicas < 1 || n_replicas > HPF_MAX_REPLICAS) return HPF_ERR_INVALID;
    for (int r = 1; r < n_replicas; ++r)
        if (params[r].n_species != params[0].n_species ||
            params[r].field_every != params[0].field_every ||
            params[r].sort_every != params[0].sort_every ||
            params[r].force_mode != params[0].force_mode ||
            (params[r].angle_k != 0.0) != (params[0].angle_k != 0.0) ||
            (params[r].dihedral_k != 0.0) != (params[0].dihedral_k != 0.0))
            return HPF_ERR_INVALID;
    for (int r = 0; r < n_replicas; ++r)
        if (params[r].thermostat == 1 || params[r].thermostat != params[0].thermostat)
            return HPF_ERR_INVALID;  // Langevin or Andersen, the same for every replica
    hpf_batch* b = new hpf_batch();
    b->R = n_replicas;
    b->stream = (cudaStream_t)stream;
    for (int r = 0; r < n_replicas; ++r) {
        hpf_ctx* c = nullptr;
        hpf_status s = hpf_init(&params[r], stream, &c);
        if (s != HPF_OK) {
            hpf_batch_destroy(b);
            return s;
        }
        b->rep.push_back(c);
    }
    std::vector<FieldCoef> coefs(n_replicas);
    for (int r = 0; r < n_replicas; ++r) coefs[r] = b->rep[r]->coef;
    cudaError_t e = cudaMalloc(&b->d_coef, sizeof(FieldCoef) * n_replicas);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_step, sizeof(long long));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_coef, coefs.data(), sizeof(FieldCoef) * n_replicas,
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        hpf_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? HPF_ERR_NOMEM : HPF_ERR_CUDA;
    }
    b->use_graphs = b->stream != nullptr;  // no capture on the legacy default stream
    *out = b;
    return HPF_OK;
}

hpf_ctx* hpf_batch_replica(hpf_batch* b, int32_t r) {
    if (!b || r < 0 || r >= b->R) return nullptr;
    return b->rep[r];
}

hpf_status hpf_batch_energy(hpf_batch* b, double* out) {
    if (!b || !out) return HPF_ERR_INVALID;
    for (hpf_ctx* c : b->rep)
        if (c->energy_pending) return fail(c, HPF_ERR_STATE, "hpf_energy_start is pending");
    // every replica's kernels and copies first, one synchronisation after
    for (hpf_ctx* c : b->rep) {
        hpf_status s = energy_launch(c);
        if (s != HPF_OK) return s;
    }
    for (hpf_ctx* c : b->rep) {
        hpf_status s = check_flags(c);
        if (s != HPF_OK) return s;
    }
    for (size_t r = 0; r < b->rep.size(); ++r) energy_finish(b->rep[r], out + 6 * r);
    return HPF_OK;
}

hpf_status hpf_batch_use_graphs(hpf_batch* b, int32_t enable) {
    if (!b) return HPF_ERR_INVALID;
    b->use_graphs = enable != 0 && b->stream != nullptr;
    return HPF_OK;
}

hpf_status hpf_batch_destroy(hpf_batch* b) {
    if (!b) return HPF_OK;
    cudaStreamSynchronize(b->stream);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (auto* c : b->rep) hpf_destroy(c);
    cudaFree(b->d_coef);
    cudaFree(b->d_step);
    cudaGetLastError();
    delete b;
    return HPF_OK;
}

hpf_status hpf_batch_step(hpf_batch* b, int32_t n_steps) {
    if (!b) return HPF_ERR_INVALID;
    if (n_steps < 0) return bfail(b, HPF_ERR_INVALID, "n_steps must be >= 0");
    hpf_ctx* c0 = b->rep[0];
    bool lockstep = true, warp = true;
    for (auto* c : b->rep) {
        if (!c->has_state) return bfail(b, HPF_ERR_STATE, "a replica has no state");
        if (c->step != c0->step) return bfail(b, HPF_ERR_STATE, "replicas are at different steps");
        warp = warp && c->warp_mode;
        lockstep = lockstep && c->cur == c0->cur && c->dmesh == c0->dmesh;
    }
    if (!warp || !lockstep) {
        for (auto* c : b->rep) {
            hpf_status s = hpf_step(c, n_steps);
            if (s != HPF_OK) return s;
        }
        return HPF_OK;
    }
    const long long fe = c0->p.field_every;
    const int se = c0->p.sort_every;
    long long left = n_steps;
    hpf_status s;
    while (left > 0) {
        // steady state: replay two captured periods at a time
        const bool aligned = c0->step % fe == 0 && fe <= 64;
        bool steady = aligned && b->use_graphs && left >= 2 * fe && !b->rep_tile.empty();
        for (auto* c : b->rep)
            steady = steady && c->mesh_step == c->step && c->field_step != c->step &&
                     c->cur == c0->cur && c->dmesh == c0->dmesh;
        if (steady) {
            long long pairs = left / (2 * fe);
            if (se > 0) {
                const long long to_sort = c0->last_sort_step + se - c0->step;
                const long long sort_pairs = to_sort > 0 ? to_sort / (2 * fe) : 0;
                if (sort_pairs < pairs) pairs = sort_pairs;
            }
            if (pairs > 0) {
                if (!b->gexec || b->graph_key != batch_key(b)) {
                    if ((s = batch_capture(b)) != HPF_OK) return s;
                }
                launch_set_counter(b->d_step, c0->step, b->stream);
                for (long long q = 0; q < pairs; ++q) {
                    CUDA_TRY(c0, cudaGraphLaunch(b->gexec, b->stream));
                    c0->launches[HPF_STAGE_FIELD] += 2;
                    c0->launches[HPF_STAGE_STEP] += 2;
                    c0->launches[HPF_STAGE_OTHER] += 2;
                }
                for (auto* c : b->rep) {
                    c->obs_step = -1;
                    c->step += 2 * fe * pairs;
                    c->mesh_step = c->step;
                    c->next_zero = false;
                    c->field_valid = true;
                    c->field_step = c->step - fe;
                }
                left -= 2 * fe * pairs;
                continue;
            }
        }
        if ((s = batch_refresh(b)) != HPF_OK) return s;
        long long chunk = fe - (c0->step % fe);
        if (chunk > left) chunk = left;
        if (chunk > 64) chunk = 64;
        if (se > 0 && c0->step - c0->last_sort_step >= se)
            for (auto* c : b->rep)
                if ((s = sort_beads(c)) != HPF_OK) return s;
        bool fuse = (c0->step + chunk) % fe == 0;
        for (auto* c : b->rep) fuse = fuse && c->next_zero && c->dmesh == c0->dmesh;
        BatchStepParams p;
        fill_step_params(b, p, (int)chunk, fuse);
        {
            StageScope sc(c0, HPF_STAGE_STEP, 1);
            launch_step_warp_batch(p, batch_max_segments(b), batch_thermostat(b), b->stream);
        }
        LAUNCH_CHECK(c0);
        batch_advance(b, chunk, fuse);
        left -= chunk;
    }
    return HPF_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ learned propagator driver

namespace {

hpf_status ensure_learned(hpf_ctx* c) {
    if (c->learned) return HPF_OK;
    LearnedBufs* L = new LearnedBufs();
    const size_t M = (size_t)c->geom.nodes, S = (size_t)c->S, xs = S > 4 ? S : 4;
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMalloc(&L->Dbase, sizeof(unsigned long long) * S * M);
    e = e ? e : cudaMalloc(&L->Dp, sizeof(unsigned long long) * S * M);
    e = e ? e : cudaMalloc(&L->x, sizeof(float) * xs * M);
    e = e ? e : cudaMalloc(&L->dphi, sizeof(float) * S * M);
    e = e ? e : cudaMalloc(&L->snap, sizeof(float) * 6 * (size_t)(c->n > 0 ? c->n : 1));
    e = e ? e : cudaMalloc(&L->acc, sizeof(double) * (2 + 2 * (size_t)force_error_partials()));
    e = e ? e : cudaMallocHost(&L->h_acc, sizeof(double) * 2);
    e = e ? e : cudaMalloc(&L->G2, sizeof(float4) * S * (size_t)c->geom.gnodes);
    c->learned = L;  // freed by hpf_destroy, also after a failed allocation
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(L->Dbase);
        cudaFree(L->Dp);
        cudaFree(L->x);
        cudaFree(L->dphi);
        cudaFree(L->snap);
        cudaFree(L->acc);
        cudaFreeHost(L->h_acc);
        cudaFree(L->G2);
        delete L;
        c->learned = nullptr;
        return fail(c, e == cudaErrorMemoryAllocation ? HPF_ERR_NOMEM : HPF_ERR_CUDA,
                    "learned-propagator buffers: %s", cudaGetErrorString(e));
    }
    return HPF_OK;
}

// eps of the candidate mesh in Dp against the true density of the current
// positions, which must be the context's mesh.  Leaves the true field in force.
hpf_status judge_mesh(hpf_ctx* c, double* eps) {
    LearnedBufs* L = c->learned;
    hpf_status s;
    if (c->field_tile < 0 && (s = run_field(c)) != HPF_OK) return s;  // picks the tile
    if (L->tmap_tile != c->field_tile) {
        L->tmap_ok = c->S <= 4 && make_mesh_tensor_map(&L->tmap,
                                                       reinterpret_cast<const long long*>(L->Dp),
                                                       c->geom, c->S, c->field_tile);
        L->tmap_tile = c->field_tile;
    }
    if ((s = field_from(c, L->Dp, L->tmap, L->tmap_ok, nullptr)) != HPF_OK) return s;
    const long long n3 = 3ll * c->n;
    {
        StageScope sc(c, HPF_STAGE_OTHER, c->n > 0 ? 1 : 0);
        launch_forces(cur_state(c), c->meta, c->n, c->geom, c->G, c->sc, HPF_FORCE_FIELD,
                      c->out_f, c->stream);
    }
    if ((s = run_field(c)) != HPF_OK) return s;
    {
        StageScope sc(c, HPF_STAGE_OTHER, c->n > 0 ? 2 : 1);
        launch_forces(cur_state(c), c->meta, c->n, c->geom, c->G, c->sc, HPF_FORCE_FIELD,
                      c->out_f + n3, c->stream);
        launch_force_error(c->out_f, c->out_f + n3, n3, L->acc, c->stream);
    }
    LAUNCH_CHECK(c);
    CUDA_TRY(c, cudaMemcpyAsync(L->h_acc, L->acc, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
    if ((s = check_flags(c)) != HPF_OK) return s;
    const double e2 = L->h_acc[0], r2 = L->h_acc[1];
    *eps = r2 > 0.0 ? sqrt(e2 / r2) : (e2 > 0.0 ? INFINITY : 0.0);
    return HPF_OK;
}

// K steps with a true scatter and field refresh at every step (the plain
// update; the same launches as a context with field_every = 1), no sorting.
hpf_status plain_window(hpf_ctx* c, int K) {
    const int fe = c->p.field_every, se = c->p.sort_every;
    c->p.field_every = 1;
    c->p.sort_every = 0;
    hpf_status s = hpf_step(c, K);
    c->p.field_every = fe;
    c->p.sort_every = se;
    return s;
}

}  // namespace

extern "C" {

hpf_status hpf_density_phi(hpf_ctx* c, float* phi) {
    if (!c) return HPF_ERR_INVALID;
    if (!c->has_state) return fail(c, HPF_ERR_STATE, "no state loaded");
    if (!phi) return fail(c, HPF_ERR_INVALID, "phi is required");
    hpf_status s = scatter_current(c);
    if (s != HPF_OK) return s;
    const long long n = (long long)mesh_words(c);
    {
        StageScope sc(c, HPF_STAGE_OTHER, 1);
        launch_mesh_to_phi(mesh_buf(c, c->dmesh), n, c->ec.phi_c,
                           reinterpret_cast<float*>(c->field_stage), c->stream);
    }
    LAUNCH_CHECK(c);
    return copy_out(c, phi, c->field_stage, sizeof(float) * n);
}

hpf_status hpf_judge_density(hpf_ctx* c, const float* phi, double* eps) {
    if (!c) return HPF_ERR_INVALID;
    if (!phi || !eps) return fail(c, HPF_ERR_INVALID, "phi and eps are required");
    if (!c->has_state) return fail(c, HPF_ERR_STATE, "no state loaded");
    hpf_status s = ensure_learned(c);
    if (s != HPF_OK) return s;
    LearnedBufs* L = c->learned;
    const long long n = (long long)mesh_words(c);
    CUDA_TRY(c, cudaMemcpyAsync(L->dphi, phi, sizeof(float) * n, cudaMemcpyDefault, c->stream));
    if ((s = scatter_current(c)) != HPF_OK) return s;
    {
        StageScope sc(c, HPF_STAGE_OTHER, 1);
        launch_mesh_predict(nullptr, L->dphi, n, 1.0 / c->ec.phi_c, L->Dp, c->stream);
    }
    LAUNCH_CHECK(c);
    return judge_mesh(c, eps);
}

hpf_status hpf_learned_mode(hpf_ctx* c, int32_t in_launch) {
    if (!c) return HPF_ERR_INVALID;
    if (in_launch < 0 || in_launch > 1) return fail(c, HPF_ERR_INVALID, "in_launch must be 0 or 1");
    hpf_status s = ensure_learned(c);
    if (s != HPF_OK) return s;
    c->learned->in_launch = in_launch != 0;
    return HPF_OK;
}

hpf_status hpf_smooth_phi(hpf_ctx* c, const float* phi_in, float* phi_out, int32_t passes) {
    if (!c) return HPF_ERR_INVALID;
    if (!phi_in || !phi_out || passes < 0 || passes > 64)
        return fail(c, HPF_ERR_INVALID, "phi_in, phi_out and 0 <= passes <= 64 are required");
    const long long n = (long long)mesh_words(c);
    // work and scratch meshes in the field staging buffer (4 n floats)
    float* a = reinterpret_cast<float*>(c->field_stage);
    float* tmp = a + n;
    CUDA_TRY(c, cudaMemcpyAsync(a, phi_in, sizeof(float) * n, cudaMemcpyDefault, c->stream));
    {
        StageScope sc(c, HPF_STAGE_OTHER, 3 * passes);
        launch_smooth_phi(a, a, tmp, c->geom.mx, c->geom.my, c->geom.mz, c->S, passes, c->stream);
    }
    LAUNCH_CHECK(c);
    return copy_out(c, phi_out, a, sizeof(float) * n);
}

hpf_status hpf_judge_density_pair(hpf_ctx* c, const float* phi_cand, const float* phi_ref,
                                  double* eps) {
    if (!c) return HPF_ERR_INVALID;
    if (!phi_cand || !phi_ref || !eps)
        return fail(c, HPF_ERR_INVALID, "phi_cand, phi_ref and eps are required");
    if (!c->has_state) return fail(c, HPF_ERR_STATE, "no state loaded");
    hpf_status s = ensure_learned(c);
    if (s != HPF_OK) return s;
    LearnedBufs* L = c->learned;
    const long long n = (long long)mesh_words(c), n3 = 3ll * c->n;
    if ((s = scatter_current(c)) != HPF_OK) return s;
    if (c->field_tile < 0 && (s = run_field(c)) != HPF_OK) return s;  // picks the tile
    CUDA_TRY(c, cudaMemcpyAsync(L->dphi, phi_cand, sizeof(float) * n, cudaMemcpyDefault,
                                c->stream));
    {
        StageScope sc(c, HPF_STAGE_OTHER, 1);
        launch_mesh_predict(nullptr, L->dphi, n, 1.0 / c->ec.phi_c, L->Dp, c->stream);
    }
    CUDA_TRY(c, cudaMemcpyAsync(L->dphi, phi_ref, sizeof(float) * n, cudaMemcpyDefault,
                                c->stream));
    {
        StageScope sc(c, HPF_STAGE_OTHER, 1);
        launch_mesh_predict(nullptr, L->dphi, n, 1.0 / c->ec.phi_c, L->Dbase, c->stream);
    }
    LAUNCH_CHECK(c);
    CUtensorMap none;
    memset(&none, 0, sizeof none);
    if ((s = field_from(c, L->Dp, none, false, nullptr)) != HPF_OK) return s;
    {
        StageScope sc(c, HPF_STAGE_OTHER, c->n > 0 ? 1 : 0);
        launch_forces(cur_state(c), c->meta, c->n, c->geom, c->G, c->sc, HPF_FORCE_FIELD,
                      c->out_f, c->stream);
    }
    if ((s = field_from(c, L->Dbase, none, false, nullptr)) != HPF_OK) return s;
    {
        StageScope sc(c, HPF_STAGE_OTHER, c->n > 0 ? 2 : 1);
        launch_forces(cur_state(c), c->meta, c->n, c->geom, c->G, c->sc, HPF_FORCE_FIELD,
                      c->out_f + n3, c->stream);
        launch_force_error(c->out_f, c->out_f + n3, n3, L->acc, c->stream);
    }
    LAUNCH_CHECK(c);
    // the field of the true density back in force
    if ((s = run_field(c)) != HPF_OK) return s;
    CUDA_TRY(c, cudaMemcpyAsync(L->h_acc, L->acc, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
    if ((s = check_flags(c)) != HPF_OK) return s;
    const double e2 = L->h_acc[0], r2 = L->h_acc[1];
    *eps = r2 > 0.0 ? sqrt(e2 / r2) : (e2 > 0.0 ? INFINITY : 0.0);
    return HPF_OK;
}

hpf_status hpf_step_learned(hpf_ctx* c, hpf_prop* prop, int32_t n_windows, int32_t K, double tol,
                            hpf_learned_stats* stats) {
    if (!c) return HPF_ERR_INVALID;
    if (!prop || n_windows < 0 || K < 2 || K > 64 || !(tol >= 0.0))
        return fail(c, HPF_ERR_INVALID, "need a network, n_windows >= 0, 2 <= K <= 64, tol >= 0");
    if (c->S != 2) return fail(c, HPF_ERR_INVALID, "the propagator models two species");
    if (c->nh) return fail(c, HPF_ERR_INVALID, "learned windows run the Langevin thermostat");
    if (!prop_mesh_is(prop, c->geom))
        return fail(c, HPF_ERR_INVALID, "the network's mesh differs from the context's");
    if (!c->has_state) return fail(c, HPF_ERR_STATE, "no state loaded");
    hpf_status s = ensure_learned(c);
    if (s != HPF_OK) return s;
    LearnedBufs* L = c->learned;
    hpf_learned_stats st;
    memset(&st, 0, sizeof st);
    const long long M = c->geom.nodes, SM = 2 * M;
    const double inv_phi_c = 1.0 / c->ec.phi_c;
    for (int w = 0; w < n_windows; ++w) {
        // the window starts at a true update t: D(t) and its field
        if (c->p.sort_every > 0 && c->step - c->last_sort_step >= c->p.sort_every &&
            (s = sort_beads(c)) != HPF_OK)
            return s;
        if (!(c->field_valid && c->field_step == c->step && c->mesh_step == c->step) &&
            (s = refresh_field(c)) != HPF_OK)
            return s;
        const long long t = c->step;
        const unsigned long long* Dt = mesh_buf(c, c->dmesh);
        CUDA_TRY(c, cudaMemcpyAsync(L->Dbase, Dt, sizeof(unsigned long long) * SM,
                                    cudaMemcpyDeviceToDevice, c->stream));
        const bool have_hist = L->hist_step >= 0 && L->hist_step == t - K;
        // in plain mode after failed judgements, predict (and judge) only every
        // few windows: the network's cost is not paid while it keeps failing
        const bool skip = L->plain_mode && L->skip_left > 0;
        if (skip) L->skip_left -= 1;
        if (have_hist && !skip) {
            StageScope sc(c, HPF_STAGE_OTHER, 6);
            launch_mesh_to_phi(Dt, SM, c->ec.phi_c, L->x + SM, c->stream);
            prop_predict(prop, L->x, L->dphi, c->stream, c->dflag);
        }
        LAUNCH_CHECK(c);
        bool judged = false;
        double eps = 0.0;
        if (have_hist && !skip && !L->plain_mode) {
            // learned window: steps t .. t+K-1 on predicted densities
            CUDA_TRY(c, cudaMemcpyAsync(L->snap, cur_state(c).x, sizeof(float) * 6 * c->n,
                                        cudaMemcpyDeviceToDevice, c->stream));
            if (L->tmap_tile != c->field_tile) {
                L->tmap_ok = make_mesh_tensor_map(&L->tmap,
                                                  reinterpret_cast<const long long*>(L->Dp),
                                                  c->geom, c->S, c->field_tile);
                L->tmap_tile = c->field_tile;
            }
            if (!c->next_zero) {
                CUDA_TRY(c, cudaMemsetAsync(mesh_buf(c, c->dmesh ^ 1), 0,
                                            sizeof(unsigned long long) * SM, c->stream));
                c->next_zero = true;
            }
            if (L->in_launch && c->warp_mode && c->sc.force_mode == 0) {
                // one launch: the field of the predicted end density D(t) + dphi in
                // G2, interpolated with the field of D(t) in the step kernel
                {
                    StageScope sc(c, HPF_STAGE_OTHER, 1);
                    launch_mesh_predict(L->Dbase, L->dphi, SM, inv_phi_c, L->Dp, c->stream);
                }
                if ((s = field_from(c, L->Dp, L->tmap, L->tmap_ok, nullptr, L->G2)) != HPF_OK)
                    return s;
                if ((s = advance(c, K, true, L->G2, 0, 1.0f / (float)K)) != HPF_OK) return s;
            } else {
                for (int j = 0; j < K; ++j) {
                    if (j > 0) {
                        {
                            StageScope sc(c, HPF_STAGE_OTHER, 1);
                            launch_mesh_predict(L->Dbase, L->dphi, SM, (double)j / K * inv_phi_c,
                                                L->Dp, c->stream);
                        }
                        if ((s = field_from(c, L->Dp, L->tmap, L->tmap_ok, nullptr)) != HPF_OK)
                            return s;
                    }
                    if ((s = advance(c, 1, j == K - 1)) != HPF_OK) return s;
                }
            }
            c->field_valid = false;  // the field in force was a predicted one
            // judge the prediction for t + K against the true scatter there
            {
                StageScope sc(c, HPF_STAGE_OTHER, 1);
                launch_mesh_predict(L->Dbase, L->dphi, SM, inv_phi_c, L->Dp, c->stream);
            }
            LAUNCH_CHECK(c);
            if ((s = judge_mesh(c, &eps)) != HPF_OK) return s;
            judged = true;
            if (eps <= tol) {
                st.learned += 1;
            } else {
                // roll back to t and take the plain update instead
                st.rejected += 1;
                CUDA_TRY(c, cudaMemcpyAsync(cur_state(c).x, L->snap, sizeof(float) * 6 * c->n,
                                            cudaMemcpyDeviceToDevice, c->stream));
                c->step = t;
                c->field_valid = false;
                c->mesh_step = -1;
                c->part_step = -1;
                c->next_zero = false;
                if ((s = plain_window(c, K)) != HPF_OK) return s;
                L->plain_mode = true;
                L->backoff = 1;
                L->skip_left = 1;
            }
        } else {
            if ((s = plain_window(c, K)) != HPF_OK) return s;
            st.plain += 1;
            if (have_hist && !skip) {
                // shadow judge of the prediction made at t
                if (c->mesh_step != c->step && (s = scatter_current(c)) != HPF_OK) return s;
                {
                    StageScope sc(c, HPF_STAGE_OTHER, 1);
                    launch_mesh_predict(L->Dbase, L->dphi, SM, inv_phi_c, L->Dp, c->stream);
                }
                LAUNCH_CHECK(c);
                if ((s = judge_mesh(c, &eps)) != HPF_OK) return s;
                judged = true;
                if (eps <= tol) {
                    L->plain_mode = false;
                    L->backoff = 0;
                } else {
                    L->backoff = L->backoff > 0 ? (L->backoff < 32 ? 2 * L->backoff : 64) : 1;
                    L->skip_left = L->backoff;
                }
            }
        }
        if (judged) {
            st.judged += 1;
            st.eps_last = eps;
            st.eps_sum += eps;
            if (eps > st.eps_max) st.eps_max = eps;
        }
        // phi(t) becomes the history of the next window
        {
            StageScope sc(c, HPF_STAGE_OTHER, 1);
            launch_mesh_to_phi(L->Dbase, SM, c->ec.phi_c, L->x, c->stream);
        }
        LAUNCH_CHECK(c);
        L->hist_step = t;
        if ((s = check_flags(c)) != HPF_OK) return s;
        st.windows += 1;
        st.steps += K;
    }
    if (stats) *stats = st;
    return HPF_OK;
}

}  // extern "C"
