// Batched launches: several contexts (uneven meshes, their own ensemble widths, time
// steps and traction tables) advanced together, either by one kernel per step whose
// time loop is captured in a CUDA graph, or by one persistent cooperative kernel with a
// bounded grid barrier between steps. An autotuner picks the mode and block shape by
// timing each on the members' own data.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ens_ctx.cuh"

using namespace ens;

struct ens_batch {
    std::vector<ens_ctx *> m;
    int form = 0;
    int mode = ENS_BATCH_GRAPH;
    int block = 256;
    int graph_steps = 20;
    int coop_grid[2] = {0, 0};  // co-resident blocks of the persistent kernel (256, 128)
    float mode_us[5] = {0, 0, 0, 0, 0};
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    std::string err;
    // device data (allocated through member 0's allocator)
    void *mem_d = nullptr;
    int4 *items_d[2] = {nullptr, nullptr};  // tiles for 256- and 128-thread blocks
    int32_t n_items[2] = {0, 0};
    int64_t **ctrs_d = nullptr;
    int *flags = nullptr;
    unsigned *bar = nullptr;
    int *h_flags = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // per block shape
    cudaGraphExec_t seq_graph = nullptr;             // sequence mode
    std::vector<uintptr_t> seq_key;
};

namespace {

int bfail(ens_batch *b, int code, const char *msg, cudaError_t e = cudaSuccess) {
    if (b) {
        b->err = std::string(ens_error_string(code)) + ": " + msg;
        if (e != cudaSuccess) b->err += std::string(" (") + cudaGetErrorString(e) + ")";
    }
    return code;
}

#define BCK(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return bfail(b, ENS_ERR_CUDA, #call, e_);                   \
    } while (0)

int idx_of(int block) { return block == 128 ? 1 : 0; }

template <typename R>
MemberDev<R> member_of(ens_ctx *c, bool tuning) {
    MemberDev<R> d{};
    d.fv.rowptr = c->rowptr;
    d.fv.ent = c->ent;
    d.fv.kc = (const R *)c->kc;
    d.fv.eh = (const R *)c->eh;
    d.fv.N = c->N;
    d.fv.Sp = c->Sp;
    d.fv.Q = c->Q;
    d.ug[0] = (const R *)c->ug[0];
    d.ug[1] = (const R *)c->ug[1];
    d.utail = c->utail;
    d.v64 = c->v64;
    d.ulo = c->ulo;
    d.v32 = c->v32;
    d.minv = (const R *)c->minv;
    d.fix = c->fix;
    d.modes = (const R *)c->modes;
    d.amp = (const R *)c->amp;
    d.step_ctr = c->step_ctr;
    d.J = tuning ? 0 : c->J;  // timing runs apply no load
    d.cur = c->cur;
    d.first = (!tuning && !c->started) ? 1 : 0;
    const double beta = 0.5 * c->alpha * c->dt;
    d.c1 = (1.0 - beta) / (1.0 + beta);
    d.c2 = c->dt / (1.0 + beta);
    d.c1s = 1.0 - beta;
    d.c2s = 0.5 * c->dt;
    d.dt = c->dt;
    return d;
}

// Upload the member table (current parities, start flags, tables) before a call.
template <typename R>
int upload_members(ens_batch *b, bool tuning) {
    std::vector<MemberDev<R>> h(b->m.size());
    for (size_t k = 0; k < b->m.size(); k++) h[k] = member_of<R>(b->m[k], tuning);
    BCK(cudaMemcpyAsync(b->mem_d, h.data(), sizeof(MemberDev<R>) * h.size(), cudaMemcpyHostToDevice,
                        b->stream));
    return ENS_OK;
}

int upload(ens_batch *b, bool tuning) {
    return b->form == kFP64 ? upload_members<double>(b, tuning) : upload_members<float>(b, tuning);
}

cudaError_t step_launch(ens_batch *b, int block, int32_t k_off) {
    const int x = idx_of(block);
    if (b->form == kFP64)
        return launch_batch_step<double>(b->form, block, (const MemberDev<double> *)b->mem_d,
                                         b->items_d[x], b->n_items[x], k_off, b->flags, b->stream);
    return launch_batch_step<float>(b->form, block, (const MemberDev<float> *)b->mem_d,
                                    b->items_d[x], b->n_items[x], k_off, b->flags, b->stream);
}

cudaError_t persistent_launch(ens_batch *b, int block, int32_t n) {
    const int x = idx_of(block);
    if (b->form == kFP64)
        return launch_batch_persistent<double>(b->form, block, (const MemberDev<double> *)b->mem_d,
                                               b->items_d[x], b->n_items[x], n, b->bar, b->flags,
                                               b->coop_grid[x], b->stream);
    return launch_batch_persistent<float>(b->form, block, (const MemberDev<float> *)b->mem_d,
                                          b->items_d[x], b->n_items[x], n, b->bar, b->flags,
                                          b->coop_grid[x], b->stream);
}

// Host bookkeeping of the members after n steps.
void advance_members(ens_batch *b, int64_t n) {
    for (ens_ctx *c : b->m) {
        c->step += n;
        c->cur ^= (int)(n & 1);
        if (n > 0) c->started = true;
    }
}

// Run n steps in the given mode and shape; on return the host bookkeeping is updated and
// the step counters advanced (asynchronously).
// Sequence mode: every member's own (autotuned, staged) step kernel, back to back per
// step, with the time loop captured in a graph. The graph bakes each member's buffer
// parity, so it is rebuilt when a member's parity changed since the capture.
int run_sequence(ens_batch *b, int64_t n, bool tuning) {
    const int32_t nm = (int32_t)b->m.size();
    int64_t left = n;
    bool any_first = false;
    for (ens_ctx *c : b->m) any_first |= (!tuning && !c->started);
    if (any_first) {
        for (ens_ctx *c : b->m) BCK(ctx_launch_step(c, 0, !c->started, b->stream));
        BCK(launch_advance_many(b->ctrs_d, nm, 1, b->stream));
        advance_members(b, 1);
        left -= 1;
    }
    const int K = b->graph_steps;
    // everything the graph bakes into kernel parameters: parities and traction buffers
    std::vector<uintptr_t> key;
    for (ens_ctx *c : b->m) {
        key.push_back((uintptr_t)(c->cur & 1));
        key.push_back((uintptr_t)c->amp);
        key.push_back((uintptr_t)c->modes);
        key.push_back((uintptr_t)(tuning ? 0 : c->J));
    }
    if (left >= K && (!b->seq_graph || b->seq_key != key)) {
        if (b->seq_graph) cudaGraphExecDestroy(b->seq_graph);
        b->seq_graph = nullptr;
        cudaGraph_t g = nullptr;
        BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        std::vector<int> saved_J(nm);
        for (int32_t m = 0; m < nm; m++) {
            saved_J[m] = b->m[m]->J;
            if (tuning) b->m[m]->J = 0;  // timing runs apply no load
        }
        for (int k = 0; k < K && e == cudaSuccess; k++)
            for (int32_t m = 0; m < nm && e == cudaSuccess; m++) e = ctx_launch_step(b->m[m], k, false, b->stream);
        for (int32_t m = 0; m < nm; m++) b->m[m]->J = saved_J[m];
        if (e == cudaSuccess) e = launch_advance_many(b->ctrs_d, nm, K, b->stream);
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess)
            return bfail(b, ENS_ERR_CUDA, "sequence graph capture", e != cudaSuccess ? e : e2);
        e = cudaGraphInstantiate(&b->seq_graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(b, ENS_ERR_CUDA, "sequence graph instantiate", e);
        b->seq_key = key;
    }
    while (left >= K) {
        BCK(cudaGraphLaunch(b->seq_graph, b->stream));
        advance_members(b, K);
        left -= K;
    }
    if (left > 0) {
        std::vector<int> saved_J(nm);
        for (int32_t m = 0; m < nm; m++) {
            saved_J[m] = b->m[m]->J;
            if (tuning) b->m[m]->J = 0;
        }
        cudaError_t e = cudaSuccess;
        for (int32_t k = 0; k < (int32_t)left && e == cudaSuccess; k++)
            for (int32_t m = 0; m < nm && e == cudaSuccess; m++) e = ctx_launch_step(b->m[m], k, false, b->stream);
        for (int32_t m = 0; m < nm; m++) b->m[m]->J = saved_J[m];
        BCK(e);
        BCK(launch_advance_many(b->ctrs_d, nm, left, b->stream));
        advance_members(b, left);
    }
    return ENS_OK;
}

int run(ens_batch *b, int mode, int block, int64_t n, bool tuning) {
    if (n <= 0) return ENS_OK;
    if (mode == ENS_BATCH_SEQUENCE) return run_sequence(b, n, tuning);
    int rc = upload(b, tuning);
    if (rc != ENS_OK) return rc;
    const int32_t nm = (int32_t)b->m.size();
    bool any_first = false;
    for (ens_ctx *c : b->m) any_first |= (!tuning && !c->started);
    if (mode == ENS_BATCH_PERSISTENT) {
        int64_t done = 0;
        while (done < n) {
            const int32_t chunk = (int32_t)std::min<int64_t>(n - done, 1 << 20);
            BCK(persistent_launch(b, block, chunk));
            BCK(launch_advance_many(b->ctrs_d, nm, chunk, b->stream));
            advance_members(b, chunk);
            done += chunk;
            if (done < n) {
                rc = upload(b, tuning);
                if (rc != ENS_OK) return rc;
            }
        }
        return ENS_OK;
    }
    int64_t left = n;
    if (any_first) {  // the start step runs on its own, then every member is started
        BCK(step_launch(b, block, 0));
        BCK(launch_advance_many(b->ctrs_d, nm, 1, b->stream));
        advance_members(b, 1);
        left -= 1;
        rc = upload(b, tuning);
        if (rc != ENS_OK) return rc;
    }
    const int K = b->graph_steps;
    const int x = idx_of(block);
    if (left >= K) {
        if (!b->graph[x]) {  // capture K step launches and the counter advance once
            cudaGraph_t g = nullptr;
            BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (int k = 0; k < K && e == cudaSuccess; k++) e = step_launch(b, block, k);
            if (e == cudaSuccess) e = launch_advance_many(b->ctrs_d, nm, K, b->stream);
            cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
            if (e != cudaSuccess || e2 != cudaSuccess)
                return bfail(b, ENS_ERR_CUDA, "graph capture", e != cudaSuccess ? e : e2);
            e = cudaGraphInstantiate(&b->graph[x], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return bfail(b, ENS_ERR_CUDA, "graph instantiate", e);
        }
        while (left >= K) {  // K is even: the buffer parities are the same after a replay
            BCK(cudaGraphLaunch(b->graph[x], b->stream));
            advance_members(b, K);
            left -= K;
        }
    }
    if (left > 0) {
        for (int32_t k = 0; k < (int32_t)left; k++) BCK(step_launch(b, block, k));
        BCK(launch_advance_many(b->ctrs_d, nm, left, b->stream));
        advance_members(b, left);
    }
    return ENS_OK;
}

// Copies of every member's state, to restore after the autotuner's timing runs.
struct Backup {
    std::vector<std::vector<std::pair<void *, void *>>> bufs;  // (dst backup, src live)
    std::vector<std::vector<size_t>> bytes;
    std::vector<int64_t> step;
    std::vector<int> cur;
    std::vector<bool> started;
};

std::vector<std::pair<void *, size_t>> state_buffers(ens_ctx *c) {
    const size_t n = (size_t)c->N * 3 * c->Sp;
    const size_t es = elem_size(c->form);
    std::vector<std::pair<void *, size_t>> v = {{c->ug[0], es * n}, {c->ug[1], es * n}};
    if (c->utail) v.push_back({c->utail, 4 * n});
    if (c->v64) v.push_back({c->v64, 8 * n});
    if (c->ulo) v.push_back({c->ulo, 4 * n});
    if (c->v32) v.push_back({c->v32, 4 * n});
    v.push_back({c->step_ctr, sizeof(int64_t)});
    return v;
}

int autotune(ens_batch *b) {
    // save state
    std::vector<std::vector<std::pair<void *, size_t>>> live(b->m.size());
    std::vector<std::vector<void *>> saved(b->m.size());
    std::vector<int64_t> step0(b->m.size());
    std::vector<int> cur0(b->m.size());
    std::vector<bool> st0(b->m.size());
    int rc = ENS_OK;
    for (size_t k = 0; k < b->m.size() && rc == ENS_OK; k++) {
        ens_ctx *c = b->m[k];
        live[k] = state_buffers(c);
        for (auto &pr : live[k]) {
            void *p = ctx_alloc(c, pr.second);
            if (!p) {
                rc = bfail(b, ENS_ERR_ALLOC, "autotune state backup");
                break;
            }
            saved[k].push_back(p);
            cudaError_t e = cudaMemcpyAsync(p, pr.first, pr.second, cudaMemcpyDeviceToDevice, b->stream);
            if (e != cudaSuccess) rc = bfail(b, ENS_ERR_CUDA, "autotune backup copy", e);
        }
        step0[k] = c->step;
        cur0[k] = c->cur;
        st0[k] = c->started;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == ENS_OK) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        const int modes[5] = {ENS_BATCH_GRAPH, ENS_BATCH_GRAPH, ENS_BATCH_PERSISTENT,
                              ENS_BATCH_PERSISTENT, ENS_BATCH_SEQUENCE};
        const int blocks[5] = {256, 128, 256, 128, 0};
        float best = -1.0f;
        const int steps = 2 * b->graph_steps;
        for (int v = 0; v < 5 && rc == ENS_OK; v++) {
            if (modes[v] == ENS_BATCH_PERSISTENT && b->coop_grid[idx_of(blocks[v])] <= 0) {
                b->mode_us[v] = -1.0f;
                continue;
            }
            rc = run(b, modes[v], blocks[v], b->graph_steps, true);  // warm-up (captures the graph)
            if (rc != ENS_OK) break;
            cudaEventRecord(e0, b->stream);
            rc = run(b, modes[v], blocks[v], steps, true);
            if (rc != ENS_OK) break;
            cudaEventRecord(e1, b->stream);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                rc = bfail(b, ENS_ERR_CUDA, "autotune timing", e);
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            b->mode_us[v] = 1000.0f * ms / steps;
            if (best < 0.0f || b->mode_us[v] < best) {
                best = b->mode_us[v];
                b->mode = modes[v];
                b->block = blocks[v];
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    // restore state (also after a failure)
    for (size_t k = 0; k < b->m.size(); k++) {
        for (size_t j = 0; j < saved[k].size(); j++)
            cudaMemcpyAsync(live[k][j].first, saved[k][j], live[k][j].second, cudaMemcpyDeviceToDevice,
                            b->stream);
    }
    cudaStreamSynchronize(b->stream);
    for (size_t k = 0; k < b->m.size(); k++) {
        for (void *p : saved[k]) ctx_free(b->m[k], p);
        if (k < step0.size()) {
            b->m[k]->step = step0[k];
            b->m[k]->cur = cur0[k];
            b->m[k]->started = st0[k];
        }
    }
    if (rc == ENS_OK) {
        BCK(cudaMemcpyAsync(b->h_flags, b->flags, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
        BCK(cudaStreamSynchronize(b->stream));
        if (b->h_flags[0] & 2) return bfail(b, ENS_ERR_TIMEOUT, "autotune: a grid barrier gave up");
        BCK(cudaMemsetAsync(b->flags, 0, 4 * sizeof(int), b->stream));
    }
    return rc;
}

}  // namespace

extern "C" {

void ens_batch_destroy(ens_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto &g : b->graph)
        if (g) cudaGraphExecDestroy(g);
    if (b->seq_graph) cudaGraphExecDestroy(b->seq_graph);
    if (!b->m.empty()) {
        ens_ctx *c0 = b->m[0];
        ctx_free(c0, b->mem_d);
        ctx_free(c0, b->items_d[0]);
        ctx_free(c0, b->items_d[1]);
        ctx_free(c0, b->ctrs_d);
        ctx_free(c0, b->flags);
        ctx_free(c0, b->bar);
    }
    if (b->h_flags) cudaFreeHost(b->h_flags);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char *ens_batch_last_error(const ens_batch *b) { return b ? b->err.c_str() : ""; }

int ens_batch_create(ens_ctx *const *members, int32_t n, int32_t mode, ens_batch **out) {
    if (!out) return ENS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!members || n < 1 || mode < ENS_BATCH_AUTO || mode > ENS_BATCH_SEQUENCE)
        return ENS_ERR_INVALID_ARG;
    for (int32_t k = 0; k < n; k++) {
        if (!members[k]) return ENS_ERR_INVALID_ARG;
        for (int32_t j = 0; j < k; j++)
            if (members[j] == members[k]) return ENS_ERR_INVALID_ARG;
        if (members[k]->form != members[0]->form || members[k]->device != members[0]->device)
            return ENS_ERR_INVALID_ARG;
        if (members[k]->peak || members[k]->geo_k) return ENS_ERR_STATE;  // per-context features only
    }
    ens_batch *b = new (std::nothrow) ens_batch();
    if (!b) return ENS_ERR_ALLOC;
    b->m.assign(members, members + n);
    b->form = members[0]->form;
    int rc = [&]() -> int {
        ens_ctx *c0 = b->m[0];
        BCK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        BCK(cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming));
        BCK(cudaMallocHost((void **)&b->h_flags, 4 * sizeof(int)));
        const size_t msz = b->form == kFP64 ? sizeof(MemberDev<double>) : sizeof(MemberDev<float>);
        b->mem_d = ctx_alloc(c0, msz * n);
        b->ctrs_d = (int64_t **)ctx_alloc(c0, sizeof(int64_t *) * n);
        b->flags = (int *)ctx_alloc(c0, 4 * sizeof(int));
        b->bar = (unsigned *)ctx_alloc(c0, sizeof(unsigned));
        if (!b->mem_d || !b->ctrs_d || !b->flags || !b->bar)
            return bfail(b, ENS_ERR_ALLOC, "batch tables");
        std::vector<int64_t *> ctrs(n);
        for (int32_t k = 0; k < n; k++) ctrs[k] = b->m[k]->step_ctr;
        BCK(cudaMemcpyAsync(b->ctrs_d, ctrs.data(), sizeof(int64_t *) * n, cudaMemcpyHostToDevice,
                            b->stream));
        BCK(cudaMemsetAsync(b->flags, 0, 4 * sizeof(int), b->stream));
        // tiles of about 1024 node-samples: BLOCK / Qt nodes x Qt lanes per tile
        const int blocks[2] = {256, 128};
        for (int x = 0; x < 2; x++) {
            std::vector<int4> items;
            for (int32_t k = 0; k < n; k++) {
                ens_ctx *c = b->m[k];
                const int32_t Qt = std::min(c->Q, blocks[x]);
                const int32_t nbt = blocks[x] / Qt;
                for (int32_t n0 = 0; n0 < c->N; n0 += nbt)
                    for (int32_t q0 = 0; q0 < c->Q; q0 += Qt) items.push_back(make_int4(k, n0, q0, 0));
            }
            b->n_items[x] = (int32_t)items.size();
            b->items_d[x] = (int4 *)ctx_alloc(c0, sizeof(int4) * items.size());
            if (!b->items_d[x]) return bfail(b, ENS_ERR_ALLOC, "tile table");
            BCK(cudaMemcpyAsync(b->items_d[x], items.data(), sizeof(int4) * items.size(),
                                cudaMemcpyHostToDevice, b->stream));
            b->coop_grid[x] = b->form == kFP64 ? batch_persistent_grid<double>(b->form, blocks[x])
                                               : batch_persistent_grid<float>(b->form, blocks[x]);
        }
        BCK(cudaStreamSynchronize(b->stream));
        for (ens_ctx *c : b->m) BCK(cudaStreamSynchronize(c->stream));
        if (mode == ENS_BATCH_AUTO) return autotune(b);
        b->mode = mode;
        b->block = 256;
        if (mode == ENS_BATCH_PERSISTENT && b->coop_grid[0] <= 0)
            return bfail(b, ENS_ERR_INVALID_ARG, "persistent kernel cannot be made co-resident");
        return ENS_OK;
    }();
    if (rc != ENS_OK) {
        // the batch is gone: leave the reason on the first member (ens_last_error)
        if (!b->m.empty()) b->m[0]->err = b->err;
        ens_batch_destroy(b);
        return rc;
    }
    *out = b;
    return ENS_OK;
}

int ens_batch_step(ens_batch *b, int64_t n) {
    if (!b) return ENS_ERR_INVALID_ARG;
    if (n < 0) return bfail(b, ENS_ERR_INVALID_ARG, "n < 0");
    for (ens_ctx *c : b->m) {
        if (c->J == 0) return bfail(b, ENS_ERR_STATE, "a member has no traction table");
        if (c->peak || c->geo_k)
            return bfail(b, ENS_ERR_STATE, "a member tracks a running peak or updates its geometry (not in batches)");
        if (c->step + n > c->n_amp) return bfail(b, ENS_ERR_RANGE, "a member's traction table is too short");
    }
    if (n == 0) return ENS_OK;
    // order after every member's pending work
    for (ens_ctx *c : b->m) {
        BCK(cudaEventRecord(b->ev, c->stream));
        BCK(cudaStreamWaitEvent(b->stream, b->ev, 0));
    }
    BCK(cudaMemsetAsync(b->flags, 0, sizeof(int), b->stream));
    int rc = run(b, b->mode, b->block, n, false);
    if (rc != ENS_OK) return rc;
    BCK(cudaMemcpyAsync(b->h_flags, b->flags, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    if (b->h_flags[0] & 2) return bfail(b, ENS_ERR_TIMEOUT, "a grid barrier gave up");
    if (b->h_flags[0] & 1) return bfail(b, ENS_ERR_NONFINITE, "a displacement became Inf/NaN");
    return ENS_OK;
}

int ens_batch_info(const ens_batch *b, ens_batch_info_t *info) {
    if (!b || !info) return ENS_ERR_INVALID_ARG;
    ens_batch_info_t r{};
    r.n_members = (int32_t)b->m.size();
    r.mode = b->mode;
    r.block = b->block;
    r.graph_steps = b->graph_steps;
    r.n_tiles = b->n_items[idx_of(b->block)];
    r.persistent_grid = b->coop_grid[idx_of(b->block)];
    for (int k = 0; k < 5; k++) r.mode_us[k] = b->mode_us[k];
    double bytes = 0.0;
    for (ens_ctx *c : b->m) {
        ens_info_t i{};
        ens_info(c, &i);
        bytes += i.bytes_per_step;
    }
    r.bytes_per_step = bytes;
    *info = r;
    return ENS_OK;
}

}  // extern "C"
