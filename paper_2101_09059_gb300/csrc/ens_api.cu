// Host side of the C ABI declared in include/ens.h: argument checking, the node ->
// element incidence lists, device memory, and the launch sequence of every call.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/ens.h"
#include "ens_internal.cuh"

using namespace ens;

#include "ens_ctx.cuh"

namespace {

const char *code_name(int code) {
    switch (code) {
    case ENS_OK: return "ok";
    case ENS_ERR_INVALID_ARG: return "invalid argument";
    case ENS_ERR_ALLOC: return "device allocation failed";
    case ENS_ERR_CUDA: return "CUDA runtime error";
    case ENS_ERR_UNSTABLE_DT: return "time step above the stability limit";
    case ENS_ERR_NONFINITE: return "non-finite displacement";
    case ENS_ERR_TIMEOUT: return "device wait timed out";
    case ENS_ERR_RANGE: return "step index past the end of the traction table";
    case ENS_ERR_STATE: return "call not valid in the current state";
    default: return "unknown status";
    }
}

int fail(ens_ctx *c, int code, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = std::string(code_name(code)) + ": " + buf;
    }
    return code;
}

#define CK(call)                                                                             \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(c, ENS_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

void *dev_alloc(ens_ctx *c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void *p = nullptr;
    if (c->custom_alloc) {
        p = c->al.alloc(bytes, (void *)c->stream, c->al.user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        c->bufs.emplace_back(p, bytes);
        c->buf_epoch.push_back(c->captures);
        c->held_bytes += bytes;
    }
    return p;
}

void dev_free(ens_ctx *c, void *p) {
    if (!p) return;
    for (size_t k = 0; k < c->bufs.size(); k++) {
        if (c->bufs[k].first == p) {
            size_t bytes = c->bufs[k].second;
            if (c->custom_alloc)
                c->al.release(p, bytes, (void *)c->stream, c->al.user);
            else
                cudaFree(p);
            c->held_bytes -= bytes;
            if (c->buf_epoch[k] < c->captures) c->buf_generation++;
            c->bufs.erase(c->bufs.begin() + k);
            c->buf_epoch.erase(c->buf_epoch.begin() + k);
            return;
        }
    }
}

#define ALLOC(ptr, type, count)                                                              \
    do {                                                                                     \
        ptr = (type *)dev_alloc(c, sizeof(type) * (size_t)(count));                          \
        if (!ptr)                                                                            \
            return fail(c, ENS_ERR_ALLOC, "%zu bytes for %s", sizeof(type) * (size_t)(count), \
                        #ptr);                                                               \
    } while (0)

bool finite_pos(const double *x, size_t n) {
    for (size_t k = 0; k < n; k++)
        if (!(std::isfinite(x[k]) && x[k] > 0.0)) return false;
    return true;
}

bool finite_all(const double *x, size_t n) {
    for (size_t k = 0; k < n; k++)
        if (!std::isfinite(x[k])) return false;
    return true;
}


// Algorithmic HBM bytes of one step: per node-sample the state traffic of the form
// (u read + write, v read + write, (E h) of the E/N incident elements, 1/m), plus the
// sample-independent geometry, incidence lists and traction patterns.
double bytes_per_step(const ens_ctx *c) {
    double per_ns = c->form == kFP64 ? 120.0 : (c->form == kFP32Force ? 108.0 : 84.0);
    double ns = (double)c->N * c->S * per_ns;
    double fixed = (double)c->E * 64.0 + (double)c->N * (12.0 + 24.0 * (c->J > 0 ? c->J : 1));
    return ns + fixed;
}


// Launch step k of a chunk whose first step reads buffer c->cur (the context is not
// changed): reads ug[cur ^ (k & 1)], writes the other buffer; start = Taylor start step.
cudaError_t launch_chunk_step(ens_ctx *c, int32_t k, bool start, cudaStream_t s) {
    const double beta = 0.5 * c->alpha * c->dt;
    double c1, c2;
    if (start) {  // Taylor start: v_{1/2} = (1 - beta) v_0 + dt/2 a_0
        c1 = 1.0 - beta;
        c2 = 0.5 * c->dt;
    } else {
        c1 = (1.0 - beta) / (1.0 + beta);
        c2 = c->dt / (1.0 + beta);
    }
    const int par = c->cur ^ (k & 1);
    cudaError_t e;
    if (c->form == kFP64) {
        StepArgs<double> a = make_args<double>(c);
        a.ug_cur = (const double *)c->ug[par];
        a.ug_next = (double *)c->ug[par ^ 1];
        a.k_off = k;
        a.c1 = c1;
        a.c2 = c2;
        e = launch_step<double>(c->form, a, false, s, &c->plan);
    } else {
        StepArgs<float> a = make_args<float>(c);
        a.ug_cur = (const float *)c->ug[par];
        a.ug_next = (float *)c->ug[par ^ 1];
        a.k_off = k;
        a.c1 = c1;
        a.c2 = c2;
        a.c1f = (float)c1;
        a.c2f = (float)c2;
        e = launch_step<float>(c->form, a, false, s, &c->plan);
    }
    if (e == cudaSuccess && c->peak)  // running peak of the state just written
        e = launch_peak(c->form, c->ug[par ^ 1], c->form == kFP32Force ? (const void *)c->utail : c->ulo, c->N,
                        c->Sp, c->step_ctr, k, c->peak_stride, c->peak, s);
    return e;
}

int run_steps(ens_ctx *c, int64_t n) {
    const cudaError_t stale = cudaGetLastError();
    if (stale != cudaSuccess)
        return fail(c, ENS_ERR_CUDA, "error pending before the step launches: %s",
                    cudaGetErrorString(stale));
    const int cur0 = c->cur;
    for (int64_t k = 0; k < n; k++) {
        const cudaError_t e = launch_chunk_step(c, (int32_t)k, !c->started && k == 0, c->stream);
        if (e != cudaSuccess) {
            c->cur = cur0 ^ (int)(k & 1);
            return fail(c, ENS_ERR_CUDA, "step launch (variant staged=%d block=%d): %s [%s]",
                        c->plan.staged, c->plan.block, cudaGetErrorString(e), last_launch_note());
        }
    }
    c->cur = cur0 ^ (int)(n & 1);
    return ENS_OK;
}

// Staged launch plan for `block` threads per block (nodes per block, most incidences of
// any block, shared-memory size). Returns an unstaged plan when the shape does not apply
// (threads per node do not divide the block, or the staging does not fit).
int make_stage_plan(ens_ctx *c, const std::vector<int32_t> &rowptr, int32_t block,
                    int32_t minb, StagePlan *out, int32_t vw = 0) {
    StagePlan p{};
    p.block = block;
    p.minb = minb;
    p.vw = vw > 0 ? vw : (c->form == kFP64 ? Vw<double>::V : Vw<float>::V);
    *out = p;
    const int32_t N = c->N, Sp = c->Sp;
    const int32_t Q = Sp / p.vw;
    if (Q <= 0 || Q > block || (block % Q) != 0) return ENS_OK;
    const int32_t nb = block / Q;
    const size_t es = elem_size(c->form);
    const int32_t KS = c->form == kFP64 ? 18 : 20;
    int32_t cmax = 0;
    for (int64_t n0 = 0; n0 < N; n0 += nb) {
        const int64_t n1 = std::min<int64_t>(N, n0 + nb);
        cmax = std::max<int32_t>(cmax, rowptr[n1] - rowptr[n0]);
    }
    const size_t bytes = 16 + (size_t)cmax * (16 + KS * es) + (size_t)nb * 3 * Sp * es;
    if (bytes > 160 * 1024) return ENS_OK;
    p.staged = 1;
    p.nb = nb;
    p.cnt_max = cmax;
    p.smem = (uint32_t)((bytes + 127) / 128 * 128);
    // one staging buffer without the barrier: entries, coupling blocks, own rows
    p.stage = (uint32_t)(((bytes - 16) + 127) / 128 * 128);
    *out = p;
    return ENS_OK;
}

// The fixed-stride block-record form of a staged plan (binary32 forms; the record
// pointers are filled in once the records exist).
StagePlan record_plan(StagePlan p) {
    if (!p.staged) return p;
    p.rec = 1;
    p.rec_h = (p.nb + 1 + 3) / 4;
    p.smem += 16u * (uint32_t)p.rec_h;
    p.smem = (p.smem + 127u) / 128u * 128u;
    if (p.smem > 160 * 1024) p.staged = 0;
    return p;
}

// The pipelined (persistent, double-buffered) form of a staged plan.
StagePlan pipelined_plan(StagePlan p) {
    if (!p.staged) return p;
    p.pipelined = 1;
    p.smem = 16 + 2 * p.stage;
    if (p.smem > 160 * 1024) p.staged = 0;
    return p;
}

constexpr int kTuneSteps = 8;  // even: a replay leaves the ping-pong parity unchanged
constexpr int kTuneReps = 3;

// Capture n step launches (steps k = 0 .. n-1 of a chunk from the current buffer, the
// context's current plan) into an executable graph.
int capture_steps(ens_ctx *c, int n, cudaGraphExec_t *out) {
    *out = nullptr;
    if (!c->cap) CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < n && e == cudaSuccess; k++) e = launch_chunk_step(c, k, false, c->cap);
    cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return fail(c, ENS_ERR_CUDA, "step graph capture: %s [%s]", cudaGetErrorString(e), last_launch_note());
    }
    return ENS_OK;
}

// Launch-shape autotuner: time a few steps of every candidate shape on this context's
// own mesh and coefficients, with the state filled with small non-zero values, and keep
// the fastest; the state is zeroed again afterwards. Candidate 0 is the unstaged kernel.
// The timing replays captured step graphs, as ens_step does.
int autotune(ens_ctx *c, const StagePlan *cand, int n) {
    // time on non-zero data (zeros take shortcuts in some arithmetic); reset afterwards
    const int64_t ns = (int64_t)c->N * 3 * c->Sp;
    const int dbl = c->form == kFP64;
    CK(launch_fill(c->ug[0], ns, dbl, 1e-4f, 1u, c->stream));
    CK(launch_fill(c->ug[1], ns, dbl, 1e-4f, 2u, c->stream));
    // FP32-force tails: any 29-bit pattern is a valid state; zeros do the same work
    if (c->utail) CK(cudaMemsetAsync(c->utail, 0, 4 * ns, c->stream));
    if (c->v64) CK(launch_fill(c->v64, ns, 1, 1e-2f, 4u, c->stream));
    if (c->ulo) CK(launch_fill(c->ulo, ns, 0, 1e-11f, 5u, c->stream));
    if (c->v32) CK(launch_fill(c->v32, ns, 0, 1e-2f, 6u, c->stream));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int best = -1;
    float best_ms = 0.0f;
    const StagePlan keep = c->plan;
    const int saved_started = c->started;
    c->started = true;
    int rc = ENS_OK;
    for (int k = 0; k < n && rc == ENS_OK; k++) {
        if (k > 0 && !cand[k].staged) {
            c->variant_us[k] = -1.0f;
            continue;
        }
        c->plan = cand[k];
        // time the shape the way ens_step runs it: replays of a captured graph of
        // kTuneSteps step launches (one warm-up replay, then kTuneReps timed)
        cudaGraphExec_t ge = nullptr;
        rc = capture_steps(c, kTuneSteps, &ge);
        if (rc != ENS_OK) break;
        cudaError_t ce = cudaGraphLaunch(ge, c->stream);
        if (ce == cudaSuccess) ce = cudaEventRecord(e0, c->stream);
        for (int r = 0; r < kTuneReps && ce == cudaSuccess; r++) ce = cudaGraphLaunch(ge, c->stream);
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, c->stream);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        cudaGraphExecDestroy(ge);
        if (ce != cudaSuccess) {
            rc = fail(c, ENS_ERR_CUDA, "autotune timing: %s [%s]", cudaGetErrorString(ce), last_launch_note());
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        c->variant_us[k] = 1000.0f * ms / (float)(kTuneSteps * kTuneReps);
        if (best < 0 || ms < best_ms) {
            best = k;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->started = saved_started;
    c->plan = (rc == ENS_OK && best >= 0) ? cand[best] : keep;
    c->variant = best < 0 ? 1 : best;
    if (rc == ENS_OK) {
        CK(cudaStreamSynchronize(c->stream));
        CK(cudaMemcpyAsync(c->h_flags, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (c->h_flags[0] & 4) return fail(c, ENS_ERR_CUDA, "autotune: launch plan inconsistent");
        if (c->h_flags[0] & 2) return fail(c, ENS_ERR_TIMEOUT, "autotune: bounded wait gave up");
    }
    return rc;
}

const void *state_main(const ens_ctx *c) { return c->ug[c->cur]; }

// The second state word array of the binary32 forms (compensated low parts or FP32-force
// tails), nullptr for FP64.
const void *state_aux(const ens_ctx *c) {
    if (c->form == kFP32Force) return c->utail;
    return c->ulo;
}

}  // namespace

namespace ens {
int ctx_fail(ens_ctx *c, int code, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = std::string(code_name(code)) + ": " + buf;
    }
    return code;
}
void *ctx_alloc(ens_ctx *c, size_t bytes) { return dev_alloc(c, bytes); }
cudaError_t ctx_launch_step(ens_ctx *c, int32_t k, bool start, cudaStream_t s) {
    return launch_chunk_step(c, k, start, s);
}
void ctx_free(ens_ctx *c, void *p) { dev_free(c, p); }

// Re-assembly on the current state u_m: the new per-realisation blocks go to the other
// buffer, the correction takes f_int(u_m) under the old stiffness minus K_new u_m, and the
// new blocks become current.
int geometry_reassemble(ens_ctx *c) {
    const void *aux = c->form == kFP32Force ? (const void *)c->utail : (const void *)c->ulo;
    const int next = c->geo_active ? c->kcs_cur ^ 1 : c->kcs_cur;
    CK(launch_reassemble(c->form, c->xyz_d, c->tri_d, c->E, c->Sp, c->nu, c->ks, c->ug[c->cur], aux,
                         c->kcs[next], c->flags, c->stream));
    if (c->form == kFP64) {
        StepArgs<double> a = make_args<double>(c);
        a.ug_cur = (const double *)c->ug[c->cur];
        CK(launch_geo_correct<double>(a, c->geo_active ? (const double *)c->kcs[c->kcs_cur] : nullptr,
                                      (const double *)c->kcs[next], c->geo_c64, (double *)c->geo_cR, c->stream));
    } else {
        StepArgs<float> a = make_args<float>(c);
        a.ug_cur = (const float *)c->ug[c->cur];
        CK(launch_geo_correct<float>(a, c->geo_active ? (const float *)c->kcs[c->kcs_cur] : nullptr,
                                     (const float *)c->kcs[next], c->geo_c64, (float *)c->geo_cR, c->stream));
    }
    c->kcs_cur = next;
    c->geo_active = true;
    return ENS_OK;
}

// Back to the linear stiffness and a zero correction (rest, or a restored checkpoint).
int geometry_restart(ens_ctx *c) {
    c->geo_active = false;
    c->kcs_cur = 0;
    const size_t n = (size_t)c->N * 3 * c->Sp;
    CK(cudaMemsetAsync(c->geo_c64, 0, 8 * n, c->stream));
    if (c->geo_cR != c->geo_c64) CK(cudaMemsetAsync(c->geo_cR, 0, elem_size(c->form) * n, c->stream));
    return ENS_OK;
}
}  // namespace ens

extern "C" {

const char *ens_error_string(int code) { return code_name(code); }

namespace {
thread_local std::string g_create_err;  // message of this thread's last failed ens_create
}

const char *ens_last_error(const ens_ctx *c) { return c ? c->err.c_str() : g_create_err.c_str(); }

void ens_destroy(ens_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (cudaGraphExec_t g : c->graph)
        if (g) cudaGraphExecDestroy(g);
    if (c->cap) cudaStreamDestroy(c->cap);
    while (!c->bufs.empty()) dev_free(c, c->bufs.back().first);
    if (c->h_flags) cudaFreeHost(c->h_flags);
    delete c;
}

int ens_create(const ens_mesh *mesh, int32_t S, const double *E_node, const double *h_node,
               const ens_params *p, void *stream, const ens_allocator *alloc, ens_ctx **out) {
    if (!out) return ENS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!mesh || !p || !E_node || !h_node || !mesh->xyz || !mesh->tri) return ENS_ERR_INVALID_ARG;
    const int32_t N = mesh->n_nodes, E = mesh->n_elems;
    if (N < 3 || E < 1 || S < 1) return ENS_ERR_INVALID_ARG;
    if ((int64_t)N * 3 * (((int64_t)S + 3) / 4 * 4) > (int64_t)INT32_MAX * 4) return ENS_ERR_INVALID_ARG;
    if (!(p->rho > 0.0) || !(p->nu >= 0.0 && p->nu < 1.0) || !(p->kshear > 0.0) ||
        !(p->alpha >= 0.0) || !(p->dt > 0.0) || !std::isfinite(p->rho) ||
        !std::isfinite(p->kshear) || !std::isfinite(p->alpha) || !std::isfinite(p->dt) ||
        p->precision < 0 || p->precision > 2 ||
        (p->flags & ~(ENS_FLAG_NO_AUTOTUNE | ENS_FLAG_UNSTAGED | ENS_FLAG_NO_GRAPH |
                      ENS_FLAG_DEVICE_FIELDS | ENS_FLAG_ELEMENT_COEFFS | 0xf00)) != 0 ||
        ((p->flags & ENS_FLAG_DEVICE_FIELDS) && (p->flags & ENS_FLAG_ELEMENT_COEFFS)) ||
        ((p->flags >> 8) & 0xf) > kVariants)
        return ENS_ERR_INVALID_ARG;
    if (alloc && (!alloc->alloc || !alloc->release)) return ENS_ERR_INVALID_ARG;
    if (!finite_all(mesh->xyz, 3 * (size_t)N)) return ENS_ERR_INVALID_ARG;
    const bool dev_fields = (p->flags & ENS_FLAG_DEVICE_FIELDS) != 0;
    // per-element coefficients: E_node, h_node carry (E h) and (rho hbar), [E][S]
    const bool elem_coeffs = (p->flags & ENS_FLAG_ELEMENT_COEFFS) != 0;
    const int64_t f_rows = elem_coeffs ? E : N;
    if (!dev_fields && (!finite_pos(E_node, (size_t)f_rows * S) || !finite_pos(h_node, (size_t)f_rows * S)))
        return ENS_ERR_INVALID_ARG;

    ens_ctx *c = new (std::nothrow) ens_ctx();
    if (!c) return ENS_ERR_ALLOC;
    c->N = N;
    c->E = E;
    c->S = S;
    c->Sp = (S + 3) / 4 * 4;
    c->form = p->precision;
    c->Q = c->Sp / (c->form == kFP64 ? Vw<double>::V : Vw<float>::V);
    c->rho = p->rho;
    c->nu = p->nu;
    c->ks = p->kshear;
    c->alpha = p->alpha;
    c->dt = p->dt;
    c->stream = (cudaStream_t)stream;
    c->flags_in = p->flags;
    cudaGetDevice(&c->device);
    if (alloc) {
        c->al = *alloc;
        c->custom_alloc = true;
    }
    int rc = [&]() -> int {
        // ---- incidence lists (host) ----------------------------------------------
        std::vector<int32_t> cnt(N + 1, 0);
        for (int64_t e = 0; e < E; e++) {
            const int32_t *t = mesh->tri + 3 * e;
            for (int j = 0; j < 3; j++)
                if (t[j] < 0 || t[j] >= N)
                    return fail(c, ENS_ERR_INVALID_ARG, "element %lld has node id %d outside [0, %d)",
                                (long long)e, t[j], N);
            if (t[0] == t[1] || t[1] == t[2] || t[0] == t[2])
                return fail(c, ENS_ERR_INVALID_ARG, "element %lld repeats a node", (long long)e);
            for (int j = 0; j < 3; j++) cnt[t[j] + 1]++;
        }
        for (int32_t i = 0; i < N; i++) {
            if (cnt[i + 1] == 0)
                return fail(c, ENS_ERR_INVALID_ARG, "node %d belongs to no element (zero mass)", i);
            cnt[i + 1] += cnt[i];
        }
        c->nnz = 3 * (int64_t)E;
        std::vector<int32_t> rowptr(cnt), fillp(cnt.begin(), cnt.end() - 1);
        std::vector<int4> ent(c->nnz);
        std::vector<int32_t> ec2ent(3 * (size_t)E);
        for (int32_t e = 0; e < E; e++) {
            const int32_t *t = mesh->tri + 3 * (int64_t)e;
            for (int cc = 0; cc < 3; cc++) {
                int32_t i = t[cc];
                int32_t pos = fillp[i]++;
                ent[pos] = make_int4(e, t[(cc + 1) % 3], t[(cc + 2) % 3], cc);
                ec2ent[3 * (size_t)e + cc] = pos;
            }
        }
        std::vector<uint8_t> fixb(N, 0);
        if (mesh->fixed)
            for (int32_t i = 0; i < N; i++)
                for (int d = 0; d < 3; d++)
                    if (mesh->fixed[3 * (int64_t)i + d]) fixb[i] |= (uint8_t)(1u << d);

        // ---- device copies of the inputs -------------------------------------------
        const int64_t NSp = (int64_t)N * c->Sp;
        ALLOC(c->rowptr, int32_t, N + 1);
        ALLOC(c->ent, int4, c->nnz);
        ALLOC(c->fix, uint8_t, N);
        ALLOC(c->xyz_d, double, 3 * (int64_t)N);
        ALLOC(c->tri_d, int32_t, 3 * (int64_t)E);
        ALLOC(c->ec2ent_d, int32_t, 3 * (int64_t)E);
        ALLOC(c->flags, int, 4);
        ALLOC(c->step_ctr, int64_t, 1);
        CK(cudaMallocHost((void **)&c->h_flags, 4 * sizeof(int)));
        CK(cudaMemcpyAsync(c->rowptr, rowptr.data(), sizeof(int32_t) * (N + 1), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->ent, ent.data(), sizeof(int4) * c->nnz, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->fix, fixb.data(), N, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->xyz_d, mesh->xyz, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->tri_d, mesh->tri, sizeof(int32_t) * 3 * (int64_t)E, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->ec2ent_d, ec2ent.data(), sizeof(int32_t) * 3 * (int64_t)E, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemsetAsync(c->flags, 0, 4 * sizeof(int), c->stream));
        CK(cudaMemsetAsync(c->step_ctr, 0, sizeof(int64_t), c->stream));

        // padded fields (nodal, or per element with ENS_FLAG_ELEMENT_COEFFS): padding
        // samples repeat sample 0 (finite, never reported)
        const int64_t FSp = f_rows * c->Sp;
        std::vector<double> Ep, hp;
        if (!dev_fields) {
            Ep.resize((size_t)FSp);
            hp.resize((size_t)FSp);
            for (int64_t i = 0; i < f_rows; i++)
                for (int32_t s = 0; s < c->Sp; s++) {
                    int32_t src = s < S ? s : 0;
                    Ep[i * c->Sp + s] = E_node[i * S + src];
                    hp[i * c->Sp + s] = h_node[i * S + src];
                }
        }
        double *En_d, *hn_d, *kc64, *area, *laml, *lamh, *xsq, *eh64, *m64, *w2lo, *w2hi;
        int *bad;
        ALLOC(En_d, double, FSp);
        ALLOC(hn_d, double, FSp);
        ALLOC(kc64, double, 18 * c->nnz);
        ALLOC(area, double, E);
        ALLOC(laml, double, E);
        ALLOC(lamh, double, E);
        ALLOC(xsq, double, 3 * (int64_t)E);
        ALLOC(eh64, double, (int64_t)E * c->Sp);
        ALLOC(m64, double, NSp);
        ALLOC(w2lo, double, E);
        ALLOC(w2hi, double, E);
        ALLOC(bad, int, 1);
        if (dev_fields) {
            CK(cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
            CK(launch_pad_fields(E_node, N, S, c->Sp, En_d, bad, c->stream));
            CK(launch_pad_fields(h_node, N, S, c->Sp, hn_d, bad, c->stream));
            int nbad = 0;  // (checked before anything else reads the fields)
            CK(cudaMemcpyAsync(&nbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            if (nbad) return fail(c, ENS_ERR_INVALID_ARG, "%d device field values not finite and > 0", nbad);
        } else {
            CK(cudaMemcpyAsync(En_d, Ep.data(), sizeof(double) * FSp, cudaMemcpyHostToDevice, c->stream));
            CK(cudaMemcpyAsync(hn_d, hp.data(), sizeof(double) * FSp, cudaMemcpyHostToDevice, c->stream));
        }
        const int big = 0x7fffffff;
        CK(cudaMemcpyAsync(bad, &big, sizeof(int), cudaMemcpyHostToDevice, c->stream));

        // ---- set-up kernels ----------------------------------------------------------
        CK(launch_setup_elements(c->xyz_d, c->tri_d, c->ec2ent_d, E, c->nu, c->ks, kc64, area,
                                 laml, lamh, xsq, nullptr, bad, c->stream));
        if (elem_coeffs) {  // (E h) given per element; mass from the given rho hbar
            CK(cudaMemcpyAsync(eh64, En_d, sizeof(double) * FSp, cudaMemcpyDeviceToDevice, c->stream));
            CK(launch_setup_mass_elem(c->rowptr, c->ent, area, hn_d, N, c->Sp, m64, c->stream));
        } else {
            CK(launch_setup_eh(c->tri_d, En_d, hn_d, E, c->Sp, eh64, c->stream));
            CK(launch_setup_mass(c->rowptr, c->ent, area, hn_d, N, c->Sp, c->rho, m64, c->stream));
        }
        CK(launch_setup_stability(c->tri_d, eh64, m64, area, hn_d, laml, lamh, xsq, E, S, c->Sp,
                                  c->rho, elem_coeffs ? hn_d : nullptr, w2lo, w2hi, c->stream));
        const size_t es = elem_size(c->form);
        const int to_f = c->form != kFP64;
        StagePlan cand[kVariants] = {};  // every slot unstaged until a plan is built
        if (!(c->flags_in & ENS_FLAG_UNSTAGED)) {
            const int forced = ((c->flags_in >> 8) & 0xf) - 1;  // -1: none
            int rcp = make_stage_plan(c, rowptr, 256, 4, &cand[1]);
            if (rcp == ENS_OK && (!(c->flags_in & ENS_FLAG_NO_AUTOTUNE) || forced >= 0)) {
                cand[2] = cand[1];
                cand[2].minb = 3;
                rcp = make_stage_plan(c, rowptr, 128, 6, &cand[3]);
                if (rcp == ENS_OK) rcp = make_stage_plan(c, rowptr, 64, 12, &cand[4]);
                if (rcp == ENS_OK && c->form != kFP64) {  // two samples per thread: more warps
                    rcp = make_stage_plan(c, rowptr, 256, 5, &cand[5], 2);
                    if (rcp == ENS_OK) rcp = make_stage_plan(c, rowptr, 128, 10, &cand[6], 2);
                    if (rcp == ENS_OK) {  // traction loads issued before the force loop
                        rcp = make_stage_plan(c, rowptr, 128, 9, &cand[7], 2);
                        cand[7].hoist = 1;
                    }
                    // persistent CTAs with a double-buffered staging ring
                    cand[8] = pipelined_plan(cand[5]);
                    cand[9] = pipelined_plan(cand[6]);
                    // shapes 6 and 4 staged from fixed-stride block records
                    cand[10] = record_plan(cand[6]);
                    cand[11] = record_plan(cand[4]);
                    if (cand[11].nb != cand[10].nb) cand[11].staged = 0;
                    // shape 11 with more registers per thread (10 resident blocks): the
                    // binary64 update of the FP32-force form spills at 12
                    cand[12] = cand[11];
                    cand[12].minb = 10;
                }
            }
            if (rcp != ENS_OK) return rcp;
        }
        c->plan = cand[1];
        c->plan_fo = cand[1];
        c->variant = c->plan.staged ? 1 : 0;
        const int forced_v = ((c->flags_in >> 8) & 0xf) - 1;
        if (forced_v >= 0) {
            c->plan = cand[forced_v];
            c->variant = c->plan.staged ? forced_v : 0;
        }
        c->kc = dev_alloc(c, es * (size_t)c->nnz * (to_f ? 20 : 18));
        c->minv = dev_alloc(c, es * (size_t)NSp);
        if (!c->kc || !c->minv) return fail(c, ENS_ERR_ALLOC, "coefficient buffers");
        CK(launch_pack_kc(kc64, c->nnz, c->kc, to_f, c->stream));
        if (cand[10].staged) {
            const StagePlan &rp = cand[10];
            const int64_t nblk = (N + rp.nb - 1) / rp.nb;
            const int64_t words = (int64_t)rp.rec_h + rp.cnt_max;
            std::vector<int4> rec((size_t)(nblk * words), make_int4(0, 0, 0, 0));
            for (int64_t b = 0; b < nblk; b++) {
                const int64_t n0 = b * rp.nb, n1 = std::min<int64_t>(N, n0 + rp.nb);
                const int32_t pb = rowptr[n0];
                int32_t *hdr = reinterpret_cast<int32_t *>(&rec[(size_t)(b * words)]);
                for (int32_t k = 0; k <= rp.nb; k++) hdr[k] = rowptr[std::min<int64_t>(n0 + k, n1)] - pb;
                for (int32_t j = 0; j < rowptr[n1] - pb; j++) rec[(size_t)(b * words + rp.rec_h + j)] = ent[pb + j];
            }
            c->rec_ent = (int4 *)dev_alloc(c, sizeof(int4) * rec.size());
            c->rec_kc = dev_alloc(c, sizeof(float) * (size_t)nblk * rp.cnt_max * 20);
            if (!c->rec_ent || !c->rec_kc) return fail(c, ENS_ERR_ALLOC, "block records");
            CK(cudaMemcpyAsync(c->rec_ent, rec.data(), sizeof(int4) * rec.size(), cudaMemcpyHostToDevice,
                               c->stream));
            CK(launch_pack_records((const float *)c->kc, c->rowptr, N, rp.nb, rp.cnt_max, (float *)c->rec_kc,
                                   c->stream));
            CK(cudaStreamSynchronize(c->stream));  // the host records leave scope
            for (int k : {10, 11, 12}) {
                cand[k].rec_ent = c->rec_ent;
                cand[k].rec_kc = c->rec_kc;
            }
            if (c->plan.rec) c->plan = cand[c->variant];  // a forced record shape
        }
        CK(launch_convert(m64, NSp, c->minv, to_f, 1, c->stream));
        if (to_f) {
            c->eh = dev_alloc(c, es * (size_t)E * c->Sp);
            if (!c->eh) return fail(c, ENS_ERR_ALLOC, "eh buffer");
            CK(launch_convert(eh64, (int64_t)E * c->Sp, c->eh, 1, 0, c->stream));
        } else {
            c->eh = eh64;
        }
        // element-mean modulus for the stress output
        ALLOC(c->ebar, double, (int64_t)E * c->Sp);
        if (elem_coeffs)
            CK(launch_modulus_from_coeffs(eh64, hn_d, (int64_t)E * c->Sp, c->rho, c->ebar, c->stream));
        else
            CK(launch_element_mean(c->tri_d, En_d, E, c->Sp, c->ebar, c->stream));
        int hbad = 0;
        std::vector<double> h_lo(E), h_hi(E);
        CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(h_lo.data(), w2lo, sizeof(double) * E, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(h_hi.data(), w2hi, sizeof(double) * E, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        CK(cudaGetLastError());
        dev_free(c, En_d);
        dev_free(c, hn_d);
        dev_free(c, kc64);
        dev_free(c, area);
        dev_free(c, laml);
        dev_free(c, lamh);
        dev_free(c, xsq);
        dev_free(c, m64);
        dev_free(c, w2lo);
        dev_free(c, w2hi);
        dev_free(c, bad);
        if (to_f) dev_free(c, eh64);
        if (hbad != big)
            return fail(c, ENS_ERR_INVALID_ARG, "element %d has zero or non-finite area", hbad);
        double lo = 0.0, hi = 0.0;
        for (int32_t e = 0; e < E; e++) {
            lo = std::fmax(lo, h_lo[e]);
            hi = std::fmax(hi, h_hi[e]);
        }
        c->w_lo = std::sqrt(lo);
        c->w_hi = std::sqrt(hi);
        if (c->dt * c->w_lo > 2.0)
            return fail(c, ENS_ERR_UNSTABLE_DT,
                        "dt = %.6g s exceeds 2 / omega = %.6g s (omega >= %.6g rad/s)", c->dt,
                        2.0 / c->w_lo, c->w_lo);

        // ---- state at rest -------------------------------------------------------------
        const size_t srow = sizeof(float) * (size_t)N * 3 * c->Sp;
        if (c->form == kFP64) {
            c->ug[0] = dev_alloc(c, 2 * srow);
            c->ug[1] = dev_alloc(c, 2 * srow);
            ALLOC(c->v64, double, (int64_t)N * 3 * c->Sp);
        } else if (c->form == kFP32Force) {
            c->ug[0] = dev_alloc(c, srow);
            c->ug[1] = dev_alloc(c, srow);
            ALLOC(c->utail, uint32_t, (int64_t)N * 3 * c->Sp);
            ALLOC(c->v64, double, (int64_t)N * 3 * c->Sp);
        } else {
            c->ug[0] = dev_alloc(c, srow);
            c->ug[1] = dev_alloc(c, srow);
            ALLOC(c->ulo, float, (int64_t)N * 3 * c->Sp);
            ALLOC(c->v32, float, (int64_t)N * 3 * c->Sp);
        }
        if (!c->ug[0] || !c->ug[1]) return fail(c, ENS_ERR_ALLOC, "state buffers");
        ALLOC(c->stat_mean, double, 3 * (int64_t)N);
        ALLOC(c->stat_var, double, 3 * (int64_t)N);
        int rc0 = ens_reset(c);
        if (rc0 != ENS_OK) return rc0;
        if (!(c->flags_in & (ENS_FLAG_NO_AUTOTUNE | ENS_FLAG_UNSTAGED | 0xf00)) && c->plan.staged) {
            rc0 = autotune(c, cand, kVariants);
            if (rc0 != ENS_OK) return rc0;
        }
        if (!c->plan.rec && c->rec_ent) {  // the records serve no chosen shape
            dev_free(c, c->rec_ent);
            dev_free(c, c->rec_kc);
            c->rec_ent = nullptr;
            c->rec_kc = nullptr;
        }
        return ens_reset(c);
    }();
    if (rc != ENS_OK) {
        g_create_err = c->err;
        ens_destroy(c);
        return rc;
    }
    g_create_err.clear();
    *out = c;
    return ENS_OK;
}

int ens_reset(ens_ctx *c) {
    if (!c) return ENS_ERR_INVALID_ARG;
    const size_t n = (size_t)c->N * 3 * c->Sp;
    const size_t es = c->form == kFP64 ? 8 : 4;
    CK(cudaMemsetAsync(c->ug[0], 0, es * n, c->stream));
    CK(cudaMemsetAsync(c->ug[1], 0, es * n, c->stream));
    if (c->utail) CK(cudaMemsetAsync(c->utail, 0, 4 * n, c->stream));
    if (c->v64) CK(cudaMemsetAsync(c->v64, 0, 8 * n, c->stream));
    if (c->ulo) CK(cudaMemsetAsync(c->ulo, 0, 4 * n, c->stream));
    if (c->v32) CK(cudaMemsetAsync(c->v32, 0, 4 * n, c->stream));
    CK(cudaMemsetAsync(c->step_ctr, 0, sizeof(int64_t), c->stream));
    CK(cudaMemsetAsync(c->flags, 0, 4 * sizeof(int), c->stream));
    if (c->peak) CK(cudaMemsetAsync(c->peak, 0, 8 * (size_t)c->N * c->Sp, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->cur = 0;
    c->step = 0;
    c->started = false;
    c->probe_rec = 0;
    c->probe_steps.clear();
    if (c->geo_k > 0) {  // the linear stiffness until the first re-assembly
        int rc = geometry_restart(c);
        if (rc != ENS_OK) return rc;
        CK(cudaStreamSynchronize(c->stream));
    }
    return ENS_OK;
}

int ens_set_traction(ens_ctx *c, int32_t J, const double *modes, int64_t n_steps,
                     const double *amp) {
    if (!c) return ENS_ERR_INVALID_ARG;
    if (J < 1 || J > kMaxModes || !modes || !amp || n_steps < 1)
        return fail(c, ENS_ERR_INVALID_ARG, "J = %d (1..%d), n_steps = %lld", J, kMaxModes,
                    (long long)n_steps);
    const size_t nm = (size_t)J * c->N * 3, na = (size_t)n_steps * J;
    if (!finite_all(modes, nm) || !finite_all(amp, na))
        return fail(c, ENS_ERR_INVALID_ARG, "non-finite traction values");
    if (c->form != kFP64) {
        for (size_t k = 0; k < nm; k++)
            if (std::fabs(modes[k]) > 3.0e38)
                return fail(c, ENS_ERR_INVALID_ARG, "traction pattern outside the binary32 range");
        for (size_t k = 0; k < na; k++)
            if (std::fabs(amp[k]) > 3.0e38)
                return fail(c, ENS_ERR_INVALID_ARG, "traction amplitude outside the binary32 range");
    }
    const size_t es = elem_size(c->form);
    CK(cudaStreamSynchronize(c->stream));
    dev_free(c, c->modes);
    dev_free(c, c->amp);
    c->modes = c->amp = nullptr;
    c->J = 0;
    c->modes = dev_alloc(c, es * nm);
    c->amp = dev_alloc(c, es * na);
    if (!c->modes || !c->amp) return fail(c, ENS_ERR_ALLOC, "traction buffers");
    if (c->form == kFP64) {
        CK(cudaMemcpyAsync(c->modes, modes, 8 * nm, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->amp, amp, 8 * na, cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    } else {
        std::vector<float> fm(nm), fa(na);
        for (size_t k = 0; k < nm; k++) fm[k] = (float)modes[k];
        for (size_t k = 0; k < na; k++) fa[k] = (float)amp[k];
        CK(cudaMemcpyAsync(c->modes, fm.data(), 4 * nm, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->amp, fa.data(), 4 * na, cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    c->J = J;
    c->n_amp = n_steps;
    return ENS_OK;
}

int ens_set_amplitudes(ens_ctx *c, int64_t first_row, int64_t n_rows, const double *amp) {
    if (!c) return ENS_ERR_INVALID_ARG;
    if (c->J == 0) return fail(c, ENS_ERR_STATE, "no traction table (call ens_set_traction)");
    if (!amp || n_rows < 0) return fail(c, ENS_ERR_INVALID_ARG, "null amplitudes or n_rows < 0");
    if (first_row < 0 || first_row + n_rows > c->n_amp)
        return fail(c, ENS_ERR_RANGE, "rows [%lld, %lld) outside the %lld-row table",
                    (long long)first_row, (long long)(first_row + n_rows), (long long)c->n_amp);
    const size_t na = (size_t)n_rows * c->J;
    if (!finite_all(amp, na)) return fail(c, ENS_ERR_INVALID_ARG, "non-finite amplitudes");
    if (na == 0) return ENS_OK;
    if (c->form == kFP64) {
        CK(cudaMemcpyAsync((double *)c->amp + first_row * c->J, amp, 8 * na,
                           cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    } else {
        std::vector<float> fa(na);
        for (size_t k = 0; k < na; k++) {
            if (std::fabs(amp[k]) > 3.0e38)
                return fail(c, ENS_ERR_INVALID_ARG, "amplitude outside the binary32 range");
            fa[k] = (float)amp[k];
        }
        CK(cudaMemcpyAsync((float *)c->amp + first_row * c->J, fa.data(), 4 * na,
                           cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return ENS_OK;
}

namespace {
// Steps through a captured graph: kGraphSteps launches and one counter advance, replayed.
// A graph bakes buffer pointers, the launch shape and the parity of the first step. Its
// key holds those, the current geometry-update block buffer and the buffer generation
// (advanced when a buffer that a capture may have baked is released), and a graph is
// captured when no kept one has the key. Returns the number of steps done this way.
int graph_steps(ens_ctx *c, int64_t n, int64_t *done) {
    *done = 0;
    const int K = kGraphSteps;
    if (n < 2 * K || !c->started || (c->flags_in & ENS_FLAG_NO_GRAPH)) return ENS_OK;
    std::vector<uintptr_t> key = {(uintptr_t)(c->cur & 1), (uintptr_t)c->amp, (uintptr_t)c->modes,
                                  (uintptr_t)c->J, (uintptr_t)c->variant, (uintptr_t)c->plan.staged,
                                  (uintptr_t)c->peak, (uintptr_t)c->peak_stride,
                                  (uintptr_t)(c->geo_active ? c->kcs[c->kcs_cur] : nullptr),
                                  (uintptr_t)c->buf_generation};
    int slot = -1;
    for (int q = 0; q < kGraphSlots && slot < 0; q++)
        if (c->graph[q] && c->graph_key[q] == key) slot = q;
    if (slot < 0) {
        slot = c->graph_next;
        c->graph_next = (c->graph_next + 1) % kGraphSlots;
        if (c->graph[slot]) cudaGraphExecDestroy(c->graph[slot]);
        c->graph[slot] = nullptr;
        if (!c->cap) CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
        c->captures++;
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < K && e == cudaSuccess; k++) e = launch_chunk_step(c, k, false, c->cap);
        if (e == cudaSuccess) e = launch_advance(c->step_ctr, K, c->cap);
        cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(c, ENS_ERR_CUDA, "time-loop graph capture: %s",
                        cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        e = cudaGraphInstantiate(&c->graph[slot], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->graph[slot] = nullptr;
            return fail(c, ENS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
        c->graph_key[slot] = key;
    }
    while (n - *done >= K) {  // K is even: the parity is the same after every replay
        CK(cudaGraphLaunch(c->graph[slot], c->stream));
        *done += K;
    }
    return ENS_OK;
}
}  // namespace

namespace {
// Launch n >= 1 steps from the current state (the start step first if not started).
int advance(ens_ctx *c, int64_t n) {
    int64_t left = n;
    if (!c->started) {  // the start step never goes into a graph
        int rc = run_steps(c, 1);
        if (rc != ENS_OK) return rc;
        CK(launch_advance(c->step_ctr, 1, c->stream));
        c->started = true;
        left -= 1;
    }
    int64_t done = 0;  // graph replays advance the device counter themselves
    int rc = graph_steps(c, left, &done);
    if (rc != ENS_OK) return rc;
    left -= done;
    if (left > 0) {
        rc = run_steps(c, left);
        if (rc != ENS_OK) return rc;
        CK(launch_advance(c->step_ctr, left, c->stream));
    }
    return ENS_OK;
}
}  // namespace

int ens_step(ens_ctx *c, int64_t n) {
    if (!c) return ENS_ERR_INVALID_ARG;
    if (n < 0) return fail(c, ENS_ERR_INVALID_ARG, "n = %lld", (long long)n);
    if (c->J == 0) return fail(c, ENS_ERR_STATE, "no traction table (call ens_set_traction)");
    if (c->step + n > c->n_amp)
        return fail(c, ENS_ERR_RANGE, "step %lld + %lld > %lld table rows", (long long)c->step,
                    (long long)n, (long long)c->n_amp);
    if (n == 0) return ENS_OK;
    if (n > INT32_MAX) return fail(c, ENS_ERR_INVALID_ARG, "n too large for one call");
    CK(cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream));
    // with probes or a geometry update, advance in segments that end on the recording
    // and re-assembly steps
    int64_t left = n;
    while (left > 0) {
        int64_t seg = left;
        if (c->probe_stride > 0) seg = std::min(left, c->probe_stride - c->step % c->probe_stride);
        if (c->geo_k > 0) seg = std::min(seg, c->geo_k - c->step % c->geo_k);
        int rc = advance(c, seg);
        if (rc != ENS_OK) return rc;
        c->step += seg;
        left -= seg;
        rc = probe_record(c);
        if (rc != ENS_OK) return rc;
        if (c->geo_k > 0 && c->step % c->geo_k == 0) {
            rc = geometry_reassemble(c);
            if (rc != ENS_OK) return rc;
        }
    }
    CK(cudaMemcpyAsync(c->h_flags, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->h_flags[0] & 8)
        return fail(c, ENS_ERR_NONFINITE, "an element degenerated on the deformed surface before step %lld",
                    (long long)c->step);
    if (c->h_flags[0] & 4)
        return fail(c, ENS_ERR_CUDA, "a staged block found its launch plan inconsistent");
    if (c->h_flags[0] & 2)
        return fail(c, ENS_ERR_TIMEOUT, "a staged step gave up waiting for its bulk copies");
    if (c->h_flags[0] & 1)
        return fail(c, ENS_ERR_NONFINITE, "displacement became Inf/NaN before step %lld",
                    (long long)c->step);
    return ENS_OK;
}

int ens_set_geometry_update(ens_ctx *c, int32_t k) {
    if (!c) return ENS_ERR_INVALID_ARG;
    if (k < 0) return fail(c, ENS_ERR_INVALID_ARG, "k = %d", k);
    CK(cudaStreamSynchronize(c->stream));
    c->geo_k = 0;
    c->geo_active = false;
    c->kcs_cur = 0;
    if (k == 0) {
        for (int q = 0; q < 2; q++) {
            dev_free(c, c->kcs[q]);
            c->kcs[q] = nullptr;
        }
        if (c->geo_cR != c->geo_c64) dev_free(c, c->geo_cR);
        dev_free(c, c->geo_c64);
        c->geo_c64 = nullptr;
        c->geo_cR = nullptr;
        return ENS_OK;
    }
    const size_t n = (size_t)c->N * 3 * c->Sp;
    for (int q = 0; q < 2; q++)
        if (!c->kcs[q]) {
            c->kcs[q] = dev_alloc(c, elem_size(c->form) * (size_t)c->E * 27 * c->Sp);
            if (!c->kcs[q]) return fail(c, ENS_ERR_ALLOC, "per-realisation coupling blocks");
        }
    if (!c->geo_c64) {
        c->geo_c64 = (double *)dev_alloc(c, 8 * n);
        c->geo_cR = c->form == kFP64 ? (void *)c->geo_c64 : dev_alloc(c, 4 * n);
        if (!c->geo_c64 || !c->geo_cR) return fail(c, ENS_ERR_ALLOC, "geometry-update force correction");
    }
    int rc = geometry_restart(c);
    if (rc != ENS_OK) return rc;
    c->geo_k = k;
    CK(cudaStreamSynchronize(c->stream));
    return ENS_OK;
}

int ens_get_displacement_device(ens_ctx *c, double *out, int32_t layout) {
    if (!c) return ENS_ERR_INVALID_ARG;
    if (!out || (layout != ENS_LAYOUT_SNC && layout != ENS_LAYOUT_NCS))
        return fail(c, ENS_ERR_INVALID_ARG, "output pointer or layout");
    CK(launch_export(c->form, state_main(c), state_aux(c), c->N, c->S, c->Sp, out, layout, c->stream));
    return ENS_OK;
}

int ens_get_displacement(ens_ctx *c, double *out, int32_t layout) {
    if (!c) return ENS_ERR_INVALID_ARG;
    if (!out || (layout != ENS_LAYOUT_SNC && layout != ENS_LAYOUT_NCS))
        return fail(c, ENS_ERR_INVALID_ARG, "output pointer or layout");
    const size_t n = (size_t)c->N * 3 * c->S;
    if (!c->export_buf) {
        c->export_buf = (double *)dev_alloc(c, 8 * n);
        if (!c->export_buf) return fail(c, ENS_ERR_ALLOC, "export buffer");
    }
    int rc = ens_get_displacement_device(c, c->export_buf, layout);
    if (rc != ENS_OK) return rc;
    CK(cudaMemcpyAsync(out, c->export_buf, 8 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ENS_OK;
}

int ens_stats_device(ens_ctx *c, double *mean, double *var) {
    if (!c) return ENS_ERR_INVALID_ARG;
    if (!mean || !var) return fail(c, ENS_ERR_INVALID_ARG, "null output");
    CK(launch_stats(c->form, state_main(c), state_aux(c), c->N, c->S, c->Sp, mean, var, c->stream));
    return ENS_OK;
}

int ens_stats(ens_ctx *c, double *mean, double *var) {
    if (!c) return ENS_ERR_INVALID_ARG;
    if (!mean || !var) return fail(c, ENS_ERR_INVALID_ARG, "null output");
    int rc = ens_stats_device(c, c->stat_mean, c->stat_var);
    if (rc != ENS_OK) return rc;
    const size_t n = 3 * (size_t)c->N;
    CK(cudaMemcpyAsync(mean, c->stat_mean, 8 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(var, c->stat_var, 8 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ENS_OK;
}

int ens_internal_force(ens_ctx *c, const double *u, double *f) {
    if (!c) return ENS_ERR_INVALID_ARG;
    if (!u || !f) return fail(c, ENS_ERR_INVALID_ARG, "null array");
    const size_t n = (size_t)c->N * 3 * c->S, np = (size_t)c->N * 3 * c->Sp;
    if (!finite_all(u, n)) return fail(c, ENS_ERR_INVALID_ARG, "non-finite displacement");
    if (c->form != kFP64)
        for (size_t k = 0; k < n; k++)
            if (std::fabs(u[k]) >= 0x1p128)
                return fail(c, ENS_ERR_INVALID_ARG, "displacement outside the binary32 range");
    const size_t es = elem_size(c->form);
    double *in_d = (double *)dev_alloc(c, 8 * n);
    void *ug = dev_alloc(c, es * np);
    double *f_d = (double *)dev_alloc(c, 8 * np);
    int rc = ENS_OK;
    if (!in_d || !ug || !f_d) rc = fail(c, ENS_ERR_ALLOC, "force buffers");
    cudaError_t e = cudaSuccess;
    if (rc == ENS_OK) {
        e = cudaMemcpyAsync(in_d, u, 8 * n, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = launch_import(c->form, in_d, c->N, c->S, c->Sp, ug, c->stream);
        if (e == cudaSuccess) {
            if (c->form == kFP64) {
                StepArgs<double> a = make_args<double>(c);
                a.ug_cur = (const double *)ug;
                a.force_out = f_d;
                e = launch_step<double>(c->form, a, true, c->stream, &c->plan_fo);
            } else {
                StepArgs<float> a = make_args<float>(c);
                a.ug_cur = (const float *)ug;
                a.force_out = f_d;
                e = launch_step<float>(c->form, a, true, c->stream, &c->plan_fo);
            }
        }
        std::vector<double> fp;
        if (e == cudaSuccess) {
            fp.resize(np);
            e = cudaMemcpyAsync(fp.data(), f_d, 8 * np, cudaMemcpyDeviceToHost, c->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess) {
            for (size_t row = 0; row < (size_t)c->N * 3; row++)
                memcpy(f + row * c->S, fp.data() + row * c->Sp, 8 * (size_t)c->S);
        } else {
            rc = fail(c, ENS_ERR_CUDA, "internal force: %s", cudaGetErrorString(e));
        }
    }
    cudaStreamSynchronize(c->stream);
    dev_free(c, in_d);
    dev_free(c, ug);
    dev_free(c, f_d);
    return rc;
}

int ens_get_coefficients(ens_ctx *c, double *eh, double *minv) {
    if (!c) return ENS_ERR_INVALID_ARG;
    const int to_f = c->form != kFP64;
    auto fetch = [&](const void *src, int64_t rows, double *dst) -> int {
        const size_t np = (size_t)rows * c->Sp;
        std::vector<double> tmp(np);
        if (to_f) {
            std::vector<float> t32(np);
            CK(cudaMemcpyAsync(t32.data(), src, 4 * np, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            for (size_t k = 0; k < np; k++) tmp[k] = (double)t32[k];
        } else {
            CK(cudaMemcpyAsync(tmp.data(), src, 8 * np, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
        for (int64_t r = 0; r < rows; r++)
            memcpy(dst + r * c->S, tmp.data() + r * c->Sp, 8 * (size_t)c->S);
        return ENS_OK;
    };
    if (eh) {
        int rc = fetch(c->eh, c->E, eh);
        if (rc != ENS_OK) return rc;
    }
    if (minv) {
        int rc = fetch(c->minv, c->N, minv);
        if (rc != ENS_OK) return rc;
    }
    return ENS_OK;
}

int ens_get_element_matrices(ens_ctx *c, double *kelem) {
    if (!c) return ENS_ERR_INVALID_ARG;
    if (!kelem) return fail(c, ENS_ERR_INVALID_ARG, "null output");
    double *kf = (double *)dev_alloc(c, 8 * 81 * (size_t)c->E);
    double *area = (double *)dev_alloc(c, 8 * (size_t)c->E);
    int *bad = (int *)dev_alloc(c, sizeof(int));
    int rc = ENS_OK;
    if (!kf || !area || !bad) rc = fail(c, ENS_ERR_ALLOC, "element matrix buffer");
    if (rc == ENS_OK) {
        cudaError_t e = launch_setup_elements(c->xyz_d, c->tri_d, c->ec2ent_d, c->E, c->nu, c->ks,
                                              nullptr, area, nullptr, nullptr, nullptr, kf, bad,
                                              c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(kelem, kf, 8 * 81 * (size_t)c->E, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = fail(c, ENS_ERR_CUDA, "element matrices: %s", cudaGetErrorString(e));
    }
    cudaStreamSynchronize(c->stream);
    dev_free(c, kf);
    dev_free(c, area);
    dev_free(c, bad);
    return rc;
}

namespace {
struct StateHeader {
    uint64_t magic;
    int32_t N, E, S, Sp, form, started;
    int64_t step;
    int64_t reserved[3];
};
const uint64_t kMagic = 0x32534e4557435345ull;  // "ESCWENS2"

size_t state_bytes(const ens_ctx *c) {
    const size_t n = (size_t)c->N * 3 * c->Sp;
    size_t b = sizeof(StateHeader);
    if (c->form == kFP64) b += 16 * n;                // u, v
    else if (c->form == kFP32Force) b += 16 * n;      // binary32 heads, tails, v64
    else b += 12 * n;                                 // hi, lo, v
    return b;
}
}  // namespace

int ens_state_size(const ens_ctx *c, size_t *bytes) {
    if (!c || !bytes) return ENS_ERR_INVALID_ARG;
    *bytes = state_bytes(c);
    return ENS_OK;
}

int ens_get_state(ens_ctx *c, void *buf, size_t bytes) {
    if (!c) return ENS_ERR_INVALID_ARG;
    if (!buf || bytes < state_bytes(c)) return fail(c, ENS_ERR_INVALID_ARG, "buffer too small");
    StateHeader h{kMagic, c->N, c->E, c->S, c->Sp, c->form, c->started ? 1 : 0, c->step, {0, 0, 0}};
    memcpy(buf, &h, sizeof(h));
    char *p = (char *)buf + sizeof(h);
    const size_t n = (size_t)c->N * 3 * c->Sp;
    auto get = [&](const void *src, size_t b) -> int {
        CK(cudaMemcpyAsync(p, src, b, cudaMemcpyDeviceToHost, c->stream));
        p += b;
        return ENS_OK;
    };
    int rc;
    if (c->form == kFP64) {
        if ((rc = get(c->ug[c->cur], 8 * n)) || (rc = get(c->v64, 8 * n))) return rc;
    } else if (c->form == kFP32Force) {
        if ((rc = get(c->ug[c->cur], 4 * n)) || (rc = get(c->utail, 4 * n)) || (rc = get(c->v64, 8 * n)))
            return rc;
    } else {
        if ((rc = get(c->ug[c->cur], 4 * n)) || (rc = get(c->ulo, 4 * n)) || (rc = get(c->v32, 4 * n)))
            return rc;
    }
    CK(cudaStreamSynchronize(c->stream));
    return ENS_OK;
}

int ens_set_state(ens_ctx *c, const void *buf, size_t bytes) {
    if (!c) return ENS_ERR_INVALID_ARG;
    if (!buf || bytes < state_bytes(c)) return fail(c, ENS_ERR_INVALID_ARG, "buffer too small");
    StateHeader h;
    memcpy(&h, buf, sizeof(h));
    if (h.magic != kMagic || h.N != c->N || h.E != c->E || h.S != c->S || h.Sp != c->Sp ||
        h.form != c->form || h.step < 0)
        return fail(c, ENS_ERR_INVALID_ARG, "state written by a different context layout");
    const char *p = (const char *)buf + sizeof(h);
    const size_t n = (size_t)c->N * 3 * c->Sp;
    CK(cudaStreamSynchronize(c->stream));
    auto put = [&](void *dst, size_t b) -> int {
        CK(cudaMemcpyAsync(dst, p, b, cudaMemcpyHostToDevice, c->stream));
        p += b;
        return ENS_OK;
    };
    c->cur = 0;
    int rc;
    if (c->form == kFP64) {
        if ((rc = put(c->ug[0], 8 * n)) || (rc = put(c->v64, 8 * n))) return rc;
    } else if (c->form == kFP32Force) {
        if ((rc = put(c->ug[0], 4 * n)) || (rc = put(c->utail, 4 * n)) || (rc = put(c->v64, 8 * n)))
            return rc;
    } else {
        if ((rc = put(c->ug[0], 4 * n)) || (rc = put(c->ulo, 4 * n)) || (rc = put(c->v32, 4 * n)))
            return rc;
    }
    int64_t st = h.step;
    CK(cudaMemcpyAsync(c->step_ctr, &st, sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->step = h.step;
    c->started = h.started != 0;
    if (c->geo_k > 0) {  // the checkpoint holds no re-assembled stiffness
        int rc = geometry_restart(c);
        if (rc != ENS_OK) return rc;
        CK(cudaStreamSynchronize(c->stream));
    }
    return ENS_OK;
}

int ens_info(const ens_ctx *c, ens_info_t *info) {
    if (!c || !info) return ENS_ERR_INVALID_ARG;
    ens_info_t r{};
    r.n_nodes = c->N;
    r.n_elems = c->E;
    r.n_samples = c->S;
    r.n_samples_padded = c->Sp;
    r.precision = c->form;
    r.n_modes = c->J;
    r.n_steps_table = c->n_amp;
    r.step = c->step;
    r.nnz = c->nnz;
    r.dt = c->dt;
    r.omega_lower = c->w_lo;
    r.omega_upper = c->w_hi;
    r.bytes_per_step = bytes_per_step(c);
    r.device_bytes = (double)c->held_bytes;
    r.kernel_variant = c->variant;
    for (int k = 0; k < kVariants; k++) r.variant_us[k] = c->variant_us[k];
    *info = r;
    return ENS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Internal force without any allocation.
//
// ens_internal_force allocates three device buffers per call. Some callers cannot
// allocate at that point: code running inside another framework's fixed memory
// budget, real-time loops that forbid cudaMalloc (it can synchronise the device), and
// hosts that hand this library device buffers but no allocation rights. This variant
// stages through a file-scope device array instead. Its size is fixed below; every GPU
// that loads the library holds it until the process exits.
// ---------------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB per device
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
// Per-device address cache. Two host threads making their first call on one device at
// the same time may both look the address up; they store the same value, and the
// atomics make that well defined.
std::atomic<void *> g_scratch_addr[kMaxDevices];

// Device address of g_static_scratch on device `dev`, looked up once per device with
// that device current (in host code the symbol name is only a host-side stand-in).
int static_scratch(ens_ctx *c, int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(c, ENS_ERR_INVALID_ARG, "device %d", dev);
    void *cached = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (cached == nullptr) {
        int prev = -1;
        CK(cudaGetDevice(&prev));
        if (prev != dev) CK(cudaSetDevice(dev));
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (prev != dev) cudaSetDevice(prev);
        if (e != cudaSuccess || p == nullptr)
            return fail(c, ENS_ERR_CUDA, "cudaGetSymbolAddress(g_static_scratch): %s",
                        cudaGetErrorString(e));
        g_scratch_addr[dev].store(p, std::memory_order_release);
        cached = p;
    }
    *out = cached;
    return ENS_OK;
}

}  // namespace

extern "C" int ens_internal_force_noalloc(ens_ctx *c, const double *u_dev, double *f_dev) {
    if (!c) return ENS_ERR_INVALID_ARG;
    if (!u_dev || !f_dev) return fail(c, ENS_ERR_INVALID_ARG, "null device array");
    const size_t np = (size_t)c->N * 3 * c->Sp;
    const size_t gbytes = ((elem_size(c->form) * np) + 255) & ~size_t(255);
    const size_t need = gbytes + 8 * np;
    if (need > kStaticScratchBytes)
        return fail(c, ENS_ERR_INVALID_ARG,
                    "needs %zu bytes of staging (N * 3 * Sp * (%zu + 8)), above the %zu-byte "
                    "static scratch; use ens_internal_force",
                    need, elem_size(c->form), kStaticScratchBytes);
    cudaPointerAttributes attr{};
    CK(cudaPointerGetAttributes(&attr, c->ug[0]));
    void *base = nullptr;
    int rc = static_scratch(c, attr.device, &base);
    if (rc != ENS_OK) return rc;
    void *ug = base;
    double *f_pad = (double *)((char *)base + gbytes);
    CK(launch_import(c->form, u_dev, c->N, c->S, c->Sp, ug, c->stream));
    cudaError_t e;
    if (c->form == kFP64) {
        StepArgs<double> a = make_args<double>(c);
        a.ug_cur = (const double *)ug;
        a.force_out = f_pad;
        e = launch_step<double>(c->form, a, true, c->stream);
    } else {
        StepArgs<float> a = make_args<float>(c);
        a.ug_cur = (const float *)ug;
        a.force_out = f_pad;
        e = launch_step<float>(c->form, a, true, c->stream);
    }
    if (e != cudaSuccess) return fail(c, ENS_ERR_CUDA, "force launch: %s", cudaGetErrorString(e));
    CK(cudaMemcpy2DAsync(f_dev, sizeof(double) * c->S, f_pad, sizeof(double) * c->Sp,
                         sizeof(double) * c->S, (size_t)c->N * 3, cudaMemcpyDeviceToDevice,
                         c->stream));
    return ENS_OK;
}

// ---------------------------------------------------------------------------------
// Merging ensemble statistics of sample shards (one shard per GPU or process).
// ---------------------------------------------------------------------------------
extern "C" int ens_merge_stats(int32_t n_parts, const int64_t *counts, const double *const *means,
                               const double *const *vars, int64_t n, double *mean_out,
                               double *var_out) {
    if (n_parts < 1 || !counts || !means || !vars || n < 0 || !mean_out || !var_out)
        return ENS_ERR_INVALID_ARG;
    int64_t total = 0;
    for (int32_t k = 0; k < n_parts; k++) {
        if (counts[k] < 0 || (counts[k] > 0 && (!means[k] || !vars[k]))) return ENS_ERR_INVALID_ARG;
        total += counts[k];
    }
    if (total < 1) return ENS_ERR_INVALID_ARG;
    for (int64_t i = 0; i < n; i++) {
        double mu = 0.0;
        for (int32_t k = 0; k < n_parts; k++)
            if (counts[k] > 0) mu += (double)counts[k] * means[k][i];
        mu /= (double)total;
        double m2 = 0.0;
        for (int32_t k = 0; k < n_parts; k++) {
            if (counts[k] == 0) continue;
            const double d = means[k][i] - mu;
            m2 += vars[k][i] * (double)(counts[k] - 1) + (double)counts[k] * d * d;
        }
        mean_out[i] = mu;
        var_out[i] = total > 1 ? m2 / (double)(total - 1) : 0.0;
    }
    return ENS_OK;
}
