// Host-side context shared by the library's translation units (not part of the ABI).
#pragma once

#include <string>
#include <utility>
#include <vector>

#include "../../include/ens.h"
#include "ens_internal.cuh"

namespace ens {
constexpr int kVariants = 13;  // launch shapes the autotuner can time (see ens_info_t)
constexpr int kGraphSteps = 32;  // steps per captured time-loop graph (even)
constexpr int kGraphSlots = 4;   // time-loop graphs kept per context
}

struct ens_ctx {
    int32_t device = 0;  // CUDA device the context was created on
    int32_t N = 0, E = 0, S = 0, Sp = 0, Q = 0, form = 0, J = 0;
    int64_t nnz = 0, n_amp = 0, step = 0;
    bool started = false;
    int cur = 0;
    double rho = 0, nu = 0, ks = 0, alpha = 0, dt = 0, w_lo = 0, w_hi = 0;
    cudaStream_t stream = nullptr;
    ens_allocator al{};
    bool custom_alloc = false;
    std::string err;
    size_t held_bytes = 0;
    std::vector<std::pair<void *, size_t>> bufs;
    // Kept time-loop graphs bake buffer addresses. buf_epoch[k] is the number of graph
    // captures made before bufs[k] was allocated; releasing a buffer that some capture may
    // have baked (one allocated before the latest capture) advances buf_generation, which
    // is part of every graph key, so no kept graph can name a released buffer.
    std::vector<uint64_t> buf_epoch;
    uint64_t captures = 0;
    uint64_t buf_generation = 0;

    // device data
    int32_t *rowptr = nullptr;
    int4 *ent = nullptr;
    uint8_t *fix = nullptr;
    double *xyz_d = nullptr;
    int32_t *tri_d = nullptr;
    int32_t *ec2ent_d = nullptr;
    void *kc = nullptr, *eh = nullptr, *minv = nullptr, *modes = nullptr, *amp = nullptr;
    void *ug[2] = {nullptr, nullptr};
    uint32_t *utail = nullptr;  // FP32-force: low mantissa bits of the binary64 state
    double *v64 = nullptr;
    float *ulo = nullptr, *v32 = nullptr;
    int *flags = nullptr;
    int64_t *step_ctr = nullptr;
    double *stat_mean = nullptr, *stat_var = nullptr;
    double *export_buf = nullptr;
    int *h_flags = nullptr;  // pinned
    ens::StagePlan plan{};     // launch shape of the step kernel
    ens::StagePlan plan_fo{};  // launch shape of force-only evaluations
    int4 *rec_ent = nullptr;     // fixed-stride block records (record shapes only)
    void *rec_kc = nullptr;
    int32_t variant = 0;
    float variant_us[ens::kVariants] = {};
    int32_t flags_in = 0;
    // time-loop graphs of kGraphSteps launches + counter advance (see ens_step), the most
    // recent kGraphSlots of them with their keys; a geometry update alternates between two
    // block buffers, so it keeps two graphs in use
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph[ens::kGraphSlots] = {};
    std::vector<uintptr_t> graph_key[ens::kGraphSlots];
    int32_t graph_next = 0;  // slot replaced by the next capture
    // output statistics: element-mean modulus [E][Sp], stress operators [E][6][9] (after
    // ens_set_centerline), the quantity buffer, and the probe histories
    double *ebar = nullptr;
    double *stress_w = nullptr;
    bool has_centerline = false;
    double *qty_buf = nullptr;
    size_t qty_cap = 0;
    int32_t *probe_nodes = nullptr, *probe_elems = nullptr;
    double *probe_hu = nullptr, *probe_hs = nullptr;
    int32_t probe_stride = 0, probe_nn = 0, probe_ne = 0;
    int64_t probe_rec = 0, probe_cap = 0;
    std::vector<int64_t> probe_steps;
    // running peak of |u| per node and sample [N][Sp] (ens_set_peak)
    double *peak = nullptr;
    int32_t peak_stride = 0;
    // geometry update (ens_set_geometry_update): per-realisation corner blocks
    // [E][3][9][Sp] of the deformed surface (two buffers: old and new during a
    // re-assembly), re-assembled every geo_k steps, and the force correction
    // c = f_int(u_m) - K_m u_m [N][3][Sp] in binary64 and in the force precision.
    // Until the first re-assembly (geo_active false) the linear kernels run.
    void *kcs[2] = {nullptr, nullptr};
    int32_t kcs_cur = 0;
    bool geo_active = false;
    double *geo_c64 = nullptr;
    void *geo_cR = nullptr;
    int32_t geo_k = 0;
};


namespace ens {

// Helpers defined in ens_api.cu.
int ctx_fail(ens_ctx *c, int code, const char *fmt, ...);
void *ctx_alloc(ens_ctx *c, size_t bytes);
void ctx_free(ens_ctx *c, void *p);
// Launch step k of a chunk starting at the context's current buffer (context unchanged).
cudaError_t ctx_launch_step(ens_ctx *c, int32_t k, bool start, cudaStream_t s);
// Record the probes if the current step is due (ens_outputs.cu).
int probe_record(ens_ctx *c);
// Re-assemble the per-realisation coupling blocks on the current state (ens_api.cu).
int geometry_reassemble(ens_ctx *c);
int geometry_restart(ens_ctx *c);
inline size_t elem_size(int form) { return form == kFP64 ? 8 : 4; }

template <typename R>
StepArgs<R> make_args(ens_ctx *c) {
    StepArgs<R> a{};
    a.fv.rowptr = c->rowptr;
    a.fv.ent = c->ent;
    a.fv.kc = (const R *)c->kc;
    a.fv.eh = (const R *)c->eh;
    a.fv.N = c->N;
    a.fv.Sp = c->Sp;
    a.fv.Q = c->Q;
    a.utail = c->utail;
    a.v64 = c->v64;
    a.ulo = c->ulo;
    a.v32 = c->v32;
    a.minv = (const R *)c->minv;
    a.fix = c->fix;
    a.modes = (const R *)c->modes;
    a.amp = (const R *)c->amp;
    a.step_ctr = c->step_ctr;
    a.J = c->J;
    a.dt = c->dt;
    a.dtf = (float)c->dt;
    a.flags = c->flags;
    a.kcs = c->geo_active ? (const R *)c->kcs[c->kcs_cur] : nullptr;
    a.kcorr = c->geo_active ? (const R *)c->geo_cR : nullptr;
    return a;
}

}  // namespace ens
