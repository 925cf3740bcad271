// Device Matérn random-field sampler (Section 2.1): x = K^-1 C~^(1/2) z with
// K = kappa^2 C~ + G, all S right-hand sides at once by Jacobi-preconditioned conjugate
// gradients, vectors stored [N][Sp] with the sample index innermost (Sp = S rounded up
// to even; each thread owns one node row and two samples).
//
// One CG iteration is five kernels:
//   spmv_dot   q = K p, and per-block partial sums of p.q for every sample;
//   fin_alpha  alpha_s = rz_s / (p.q)_s (0 once sample s has converged);
//   update     x += alpha p, r -= alpha q, z = M^-1 r, partial sums of r.z and r.r;
//   fin_beta   beta_s = rz_new / rz, convergence test ||r|| <= rtol ||b||, active count;
//   pupdate    p = z + beta p.
// Every reduction has a fixed shape (fixed grid, fixed tree), so results are bitwise
// reproducible; a converged sample takes alpha = beta = 0 from then on, so stopping a
// few iterations later changes nothing. Iterations run as replays of a captured graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gmrf.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1216;  // 152 SMs x 8: fixed reduction shape
constexpr int kGraphIters = 8;

thread_local char g_create_err[256] = "";

}  // namespace

struct gmrf_ctx {
    int32_t N = 0;
    int64_t nnz = 0;
    double kappa = 0.0;
    cudaStream_t stream = nullptr;
    int device = 0;
    int32_t *rowptr = nullptr, *col = nullptr;
    double *val = nullptr, *minv = nullptr, *sqrtc = nullptr;
    // work vectors, sized for cap_sp samples
    int32_t cap_sp = 0;
    double *x = nullptr, *r = nullptr, *zv = nullptr, *p = nullptr, *q = nullptr;
    double *part = nullptr;  // [2][Sp][G]: per-sample partial sums, contiguous over blocks
    double *scal = nullptr;  // [6][Sp]: rz, alpha, beta, bb, relres2, active
    int *n_active = nullptr;
    int *h_active = nullptr;  // pinned
    cudaGraphExec_t graph = nullptr;
    int32_t graph_sp = -1;
    double graph_rtol = -1.0;
    gmrf_info_t info{};
    char err[256] = "";
};

namespace {

int fail(gmrf_ctx *g, int code, const char *fmt, ...) {
    char *dst = g ? g->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return code;
}

#define CKG(call)                                                                   \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            return fail(g, GMRF_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// ---- launch geometry -------------------------------------------------------------------
// blockDim = (Qt lanes, R rows), grid = (G row-tile blocks, lane chunks); each block walks
// the row tiles blockIdx.x, blockIdx.x + G, ... so G fixes the reduction shape.
struct Geo {
    int Q, Qt, R, G, chunks;
    int64_t tiles;
};

Geo geometry(int32_t N, int32_t Sp) {
    Geo o;
    o.Q = Sp / 2;
    o.Qt = std::min(o.Q, kThreads);
    o.R = std::max(1, kThreads / o.Qt);
    o.tiles = ((int64_t)N + o.R - 1) / o.R;
    o.G = (int)std::min<int64_t>(o.tiles, kMaxBlocks);
    o.chunks = (o.Q + o.Qt - 1) / o.Qt;
    return o;
}

// Sum the per-thread double2 partials of a block over its rows (fixed pairwise tree) and
// write them to part[w][s][blockIdx.x].
__device__ __forceinline__ void block_partial(double2 v, double2 *sm, double *part, int w,
                                              int G, int32_t Sp, int lane_q) {
    const int R = blockDim.y, Qt = blockDim.x;
    const int y = threadIdx.y, xq = threadIdx.x;
    sm[y * Qt + xq] = v;
    __syncthreads();
    int p2 = 1;
    while (p2 < R) p2 <<= 1;
    for (int st = p2 >> 1; st > 0; st >>= 1) {
        if (y < st && y + st < R) {
            double2 a = sm[y * Qt + xq], b = sm[(y + st) * Qt + xq];
            sm[y * Qt + xq] = make_double2(a.x + b.x, a.y + b.y);
        }
        __syncthreads();
    }
    if (y == 0 && lane_q < Sp / 2) {
        double2 t = sm[xq];
        double *dst = part + ((size_t)w * Sp + 2 * lane_q) * G + blockIdx.x;
        dst[0] = t.x;
        dst[G] = t.y;
    }
    __syncthreads();
}

__device__ __forceinline__ double2 ld2(const double *p) { return *reinterpret_cast<const double2 *>(p); }
__device__ __forceinline__ void st2(double *p, double2 v) { *reinterpret_cast<double2 *>(p) = v; }

// r = C~^(1/2) z (padding samples 0), x = 0, z = M^-1 r, p = z; partials r.z and r.r.
__global__ void init_kernel(const double *__restrict__ zin, int32_t S, int32_t Sp, int32_t N,
                            int64_t tiles, const double *__restrict__ sqrtc,
                            const double *__restrict__ minv, double *x, double *r, double *zv,
                            double *p, double *part) {
    extern __shared__ double2 sm[];
    const int lane_q = blockIdx.y * blockDim.x + threadIdx.x;
    const bool lane_ok = lane_q < Sp / 2;
    double2 rz = make_double2(0.0, 0.0), rr = rz;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t i = t * blockDim.y + threadIdx.y;
        if (i >= N || !lane_ok) continue;
        const int s0 = 2 * lane_q;
        const double c = sqrtc[i], m = minv[i];
        const double z0 = s0 < S ? zin[i * S + s0] : 0.0;
        const double z1 = s0 + 1 < S ? zin[i * S + s0 + 1] : 0.0;
        const double2 rv = make_double2(c * z0, c * z1);
        const double2 zz = make_double2(m * rv.x, m * rv.y);
        const size_t o = (size_t)i * Sp + s0;
        st2(x + o, make_double2(0.0, 0.0));
        st2(r + o, rv);
        st2(zv + o, zz);
        st2(p + o, zz);
        rz.x += rv.x * zz.x;
        rz.y += rv.y * zz.y;
        rr.x += rv.x * rv.x;
        rr.y += rv.y * rv.y;
    }
    block_partial(rz, sm, part, 0, gridDim.x, Sp, lane_q);
    block_partial(rr, sm, part, 1, gridDim.x, Sp, lane_q);
}

// q = K p and partials of p.q.
__global__ void spmv_dot_kernel(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                const double *__restrict__ val, const double *__restrict__ p,
                                double *__restrict__ q, int32_t N, int32_t Sp, int64_t tiles,
                                double *part) {
    extern __shared__ double2 sm[];
    const int lane_q = blockIdx.y * blockDim.x + threadIdx.x;
    const bool lane_ok = lane_q < Sp / 2;
    double2 pq = make_double2(0.0, 0.0);
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t i = t * blockDim.y + threadIdx.y;
        if (i >= N || !lane_ok) continue;
        const int s0 = 2 * lane_q;
        double2 acc = make_double2(0.0, 0.0);
        const int32_t k0 = __ldg(rowptr + i), k1 = __ldg(rowptr + i + 1);
        // the first kUnroll entries: all column indices first, then all vector loads, so a
        // row costs two dependent round trips instead of one per entry
        constexpr int kUnroll = 8;
        int32_t cj[kUnroll];
        double aj[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const bool ok = k0 + u < k1;
            cj[u] = ok ? __ldg(col + k0 + u) : (int32_t)i;
            aj[u] = ok ? __ldg(val + k0 + u) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const double2 v = __ldg(reinterpret_cast<const double2 *>(p + (size_t)cj[u] * Sp + s0));
            acc.x = fma(aj[u], v.x, acc.x);
            acc.y = fma(aj[u], v.y, acc.y);
        }
        for (int32_t k = k0 + kUnroll; k < k1; k++) {
            const double a = __ldg(val + k);
            const double2 v = __ldg(reinterpret_cast<const double2 *>(p + (size_t)__ldg(col + k) * Sp + s0));
            acc.x = fma(a, v.x, acc.x);
            acc.y = fma(a, v.y, acc.y);
        }
        const size_t o = (size_t)i * Sp + s0;
        st2(q + o, acc);
        const double2 pv = ld2(p + o);
        pq.x = fma(pv.x, acc.x, pq.x);
        pq.y = fma(pv.y, acc.y, pq.y);
    }
    block_partial(pq, sm, part, 0, gridDim.x, Sp, lane_q);
}

// x += alpha p, r -= alpha q, z = M^-1 r; partials of r.z and r.r.
__global__ void update_kernel(const double *__restrict__ minv, const double *__restrict__ alpha,
                              double *x, double *r, double *zv, const double *__restrict__ p,
                              const double *__restrict__ q, int32_t N, int32_t Sp, int64_t tiles,
                              double *part) {
    extern __shared__ double2 sm[];
    const int lane_q = blockIdx.y * blockDim.x + threadIdx.x;
    const bool lane_ok = lane_q < Sp / 2;
    double2 rz = make_double2(0.0, 0.0), rr = rz;
    double2 al = make_double2(0.0, 0.0);
    if (lane_ok) al = ld2(alpha + 2 * lane_q);
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t i = t * blockDim.y + threadIdx.y;
        if (i >= N || !lane_ok) continue;
        const size_t o = (size_t)i * Sp + 2 * lane_q;
        const double2 pv = ld2(p + o), qv = ld2(q + o);
        double2 xv = ld2(x + o), rv = ld2(r + o);
        xv.x = fma(al.x, pv.x, xv.x);
        xv.y = fma(al.y, pv.y, xv.y);
        rv.x = fma(-al.x, qv.x, rv.x);
        rv.y = fma(-al.y, qv.y, rv.y);
        const double m = minv[i];
        const double2 zz = make_double2(m * rv.x, m * rv.y);
        st2(x + o, xv);
        st2(r + o, rv);
        st2(zv + o, zz);
        rz.x = fma(rv.x, zz.x, rz.x);
        rz.y = fma(rv.y, zz.y, rz.y);
        rr.x = fma(rv.x, rv.x, rr.x);
        rr.y = fma(rv.y, rv.y, rr.y);
    }
    block_partial(rz, sm, part, 0, gridDim.x, Sp, lane_q);
    block_partial(rr, sm, part, 1, gridDim.x, Sp, lane_q);
}

// p = z + beta p.
__global__ void pupdate_kernel(const double *__restrict__ beta, const double *__restrict__ zv,
                               double *p, int32_t N, int32_t Sp) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n2 = (int64_t)N * Sp / 2;
    if (t >= n2) return;
    const int32_t s0 = (int32_t)(2 * (t % (Sp / 2)));
    const double2 b = ld2(beta + s0);
    const double2 zz = ld2(zv + 2 * t);
    double2 pv = ld2(p + 2 * t);
    pv.x = fma(b.x, pv.x, zz.x);
    pv.y = fma(b.y, pv.y, zz.y);
    st2(p + 2 * t, pv);
}

// Sum of part[w][s][0..G) by one warp per sample: fixed lane assignment, fixed tree.
__device__ __forceinline__ double warp_total(const double *part, int w, int G, int32_t Sp, int s) {
    const int lane = threadIdx.x & 31;
    const double *src = part + ((size_t)w * Sp + s) * G;
    double a = 0.0;
    for (int b = lane; b < G; b += 32) a += src[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}

// scal rows: 0 rz, 1 alpha, 2 beta, 3 bb, 4 relres^2, 5 active
__global__ void fin_init_kernel(const double *part, int G, int32_t Sp, double *scal, int *n_active) {
    const int s = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (s >= Sp) return;
    const double rz = warp_total(part, 0, G, Sp, s);
    const double bb = warp_total(part, 1, G, Sp, s);
    if ((threadIdx.x & 31) == 0) {
        const bool act = bb > 0.0;
        scal[0 * Sp + s] = rz;
        scal[1 * Sp + s] = 0.0;
        scal[2 * Sp + s] = 0.0;
        scal[3 * Sp + s] = bb;
        scal[4 * Sp + s] = act ? 1.0 : 0.0;
        scal[5 * Sp + s] = act ? 1.0 : 0.0;
        if (act) atomicAdd(n_active, 1);
    }
}

__global__ void fin_alpha_kernel(const double *part, int G, int32_t Sp, double *scal, int *n_active) {
    const int s = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_active = 0;
    if (s >= Sp) return;
    const double pq = warp_total(part, 0, G, Sp, s);
    if ((threadIdx.x & 31) == 0) {
        const bool act = scal[5 * Sp + s] != 0.0;
        scal[1 * Sp + s] = (act && pq > 0.0) ? scal[0 * Sp + s] / pq : 0.0;
    }
}

__global__ void fin_beta_kernel(const double *part, int G, int32_t Sp, double rtol2, double *scal,
                                int *n_active) {
    const int s = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (s >= Sp) return;
    const double rz = warp_total(part, 0, G, Sp, s);
    const double rr = warp_total(part, 1, G, Sp, s);
    if ((threadIdx.x & 31) == 0) {
        const bool act = scal[5 * Sp + s] != 0.0;
        if (act) {
            const double bb = scal[3 * Sp + s];
            const bool done = rr <= rtol2 * bb;
            scal[2 * Sp + s] = (done || !(scal[0 * Sp + s] > 0.0)) ? 0.0 : rz / scal[0 * Sp + s];
            scal[0 * Sp + s] = rz;
            scal[4 * Sp + s] = rr / bb;
            if (done) {
                scal[5 * Sp + s] = 0.0;
            } else {
                atomicAdd(n_active, 1);
            }
        } else {
            scal[2 * Sp + s] = 0.0;
        }
    }
}

__global__ void transform_kernel(const double *__restrict__ x, int32_t N, int32_t S, int32_t Sp,
                                 double scale, double mean, int lognormal, double *out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * S) return;
    const int64_t i = t / S;
    const int32_t s = (int32_t)(t - i * S);
    const double v = scale * x[i * Sp + s];
    out[t] = lognormal ? mean * exp(v) : mean + v;
}

int alloc_work(gmrf_ctx *g, int32_t Sp) {
    if (Sp <= g->cap_sp) return GMRF_OK;
    double **v[5] = {&g->x, &g->r, &g->zv, &g->p, &g->q};
    for (double **pp : v) {
        if (*pp) cudaFree(*pp);
        *pp = nullptr;
    }
    if (g->part) cudaFree(g->part);
    if (g->scal) cudaFree(g->scal);
    g->part = g->scal = nullptr;
    g->cap_sp = 0;
    const size_t n = (size_t)g->N * Sp;
    for (double **pp : v)
        if (cudaMalloc((void **)pp, 8 * n) != cudaSuccess)
            return fail(g, GMRF_ERR_ALLOC, "%zu bytes for a work vector", 8 * n);
    if (cudaMalloc((void **)&g->part, 8 * (size_t)2 * kMaxBlocks * Sp) != cudaSuccess ||
        cudaMalloc((void **)&g->scal, 8 * (size_t)6 * Sp) != cudaSuccess)
        return fail(g, GMRF_ERR_ALLOC, "reduction buffers");
    g->cap_sp = Sp;
    if (g->graph) cudaGraphExecDestroy(g->graph);
    g->graph = nullptr;
    g->graph_sp = -1;
    return GMRF_OK;
}

// One CG iteration (five launches) on g's stream.
cudaError_t launch_iteration(gmrf_ctx *g, int32_t Sp, double rtol2) {
    const Geo o = geometry(g->N, Sp);
    const dim3 grid(o.G, o.chunks), block(o.Qt, o.R);
    const size_t sm = sizeof(double2) * o.Qt * o.R;
    const int fin_blocks = (Sp + 7) / 8;
    double *alpha = g->scal + 1 * (size_t)Sp, *beta = g->scal + 2 * (size_t)Sp;
    spmv_dot_kernel<<<grid, block, sm, g->stream>>>(g->rowptr, g->col, g->val, g->p, g->q, g->N, Sp,
                                                    o.tiles, g->part);
    fin_alpha_kernel<<<fin_blocks, 256, 0, g->stream>>>(g->part, o.G, Sp, g->scal, g->n_active);
    update_kernel<<<grid, block, sm, g->stream>>>(g->minv, alpha, g->x, g->r, g->zv, g->p, g->q, g->N,
                                                  Sp, o.tiles, g->part);
    fin_beta_kernel<<<fin_blocks, 256, 0, g->stream>>>(g->part, o.G, Sp, rtol2, g->scal, g->n_active);
    const int64_t n2 = (int64_t)g->N * Sp / 2;
    pupdate_kernel<<<(unsigned)((n2 + 255) / 256), 256, 0, g->stream>>>(beta, g->zv, g->p, g->N, Sp);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int gmrf_create(int32_t n_nodes, int32_t n_elems, const double *xyz, const int32_t *tri,
                double kappa, void *stream, gmrf_ctx **out) {
    gmrf_ctx *g = nullptr;
    if (!out) return fail(g, GMRF_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    if (n_nodes < 1 || n_elems < 1 || !xyz || !tri)
        return fail(g, GMRF_ERR_INVALID_ARG, "mesh sizes or pointers");
    if (!(kappa > 0.0) || !std::isfinite(kappa)) return fail(g, GMRF_ERR_INVALID_ARG, "kappa must be > 0");
    const int32_t N = n_nodes, E = n_elems;
    // ---- assembly (host, binary64): G from barycentric gradients, lumped C~ -------------
    std::vector<double> cl(N, 0.0);
    std::vector<int32_t> cnt(N + 1, 0);
    for (int64_t e = 0; e < E; e++)
        for (int a = 0; a < 3; a++) {
            const int32_t v = tri[3 * e + a];
            if (v < 0 || v >= N)
                return fail(g, GMRF_ERR_INVALID_ARG, "element %lld has node id %d outside [0, %d)",
                            (long long)e, v, N);
            cnt[v + 1] += 3;
        }
    for (int32_t i = 0; i < N; i++) {
        if (cnt[i + 1] == 0) return fail(g, GMRF_ERR_INVALID_ARG, "node %d belongs to no element", i);
        cnt[i + 1] += cnt[i];
    }
    std::vector<int32_t> dcol(cnt[N]);
    std::vector<double> dval(cnt[N]);
    std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t e = 0; e < E; e++) {
        const int32_t *t = tri + 3 * e;
        double X[3][3];
        for (int a = 0; a < 3; a++)
            for (int k = 0; k < 3; k++) X[a][k] = xyz[3 * (int64_t)t[a] + k];
        double e1[3], e2[3], n[3];
        for (int k = 0; k < 3; k++) {
            e1[k] = X[1][k] - X[0][k];
            e2[k] = X[2][k] - X[0][k];
        }
        n[0] = e1[1] * e2[2] - e1[2] * e2[1];
        n[1] = e1[2] * e2[0] - e1[0] * e2[2];
        n[2] = e1[0] * e2[1] - e1[1] * e2[0];
        const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(nn > 0.0) || !std::isfinite(nn))
            return fail(g, GMRF_ERR_INVALID_ARG, "element %lld has zero area", (long long)e);
        const double A = 0.5 * nn;
        // gradient of the barycentric function of corner a: (n / |n|) x (X_c - X_b) / (2 A)
        double grad[3][3];
        for (int a = 0; a < 3; a++) {
            const int b = (a + 1) % 3, c = (a + 2) % 3;
            double ed[3];
            for (int k = 0; k < 3; k++) ed[k] = X[c][k] - X[b][k];
            grad[a][0] = (n[1] * ed[2] - n[2] * ed[1]) / (nn * 2.0 * A);
            grad[a][1] = (n[2] * ed[0] - n[0] * ed[2]) / (nn * 2.0 * A);
            grad[a][2] = (n[0] * ed[1] - n[1] * ed[0]) / (nn * 2.0 * A);
        }
        for (int a = 0; a < 3; a++) {
            cl[t[a]] += A / 3.0;
            for (int b = 0; b < 3; b++) {
                const int32_t pos = fill[t[a]]++;
                dcol[pos] = t[b];
                dval[pos] = A * (grad[a][0] * grad[b][0] + grad[a][1] * grad[b][1] +
                                 grad[a][2] * grad[b][2]);
            }
        }
    }
    // merge duplicate columns row by row (ascending column order), add kappa^2 C~
    std::vector<int32_t> rowptr(N + 1, 0), col;
    std::vector<double> val;
    col.reserve(cnt[N] / 2);
    val.reserve(cnt[N] / 2);
    std::vector<double> diag(N, 0.0);
    std::vector<std::pair<int32_t, double>> row;
    for (int32_t i = 0; i < N; i++) {
        row.clear();
        for (int32_t k = cnt[i]; k < cnt[i + 1]; k++) row.emplace_back(dcol[k], dval[k]);
        std::stable_sort(row.begin(), row.end(),
                         [](const std::pair<int32_t, double> &a, const std::pair<int32_t, double> &b) {
                             return a.first < b.first;
                         });
        for (size_t k = 0; k < row.size();) {
            const int32_t j = row[k].first;
            double s = 0.0;
            for (; k < row.size() && row[k].first == j; k++) s += row[k].second;
            if (j == i) {
                s += kappa * kappa * cl[i];
                diag[i] = s;
            }
            col.push_back(j);
            val.push_back(s);
        }
        rowptr[i + 1] = (int32_t)col.size();
    }
    std::vector<double> minv(N), sqrtc(N);
    for (int32_t i = 0; i < N; i++) {
        minv[i] = 1.0 / diag[i];
        sqrtc[i] = std::sqrt(cl[i]);
    }

    g = new (std::nothrow) gmrf_ctx();
    if (!g) return fail(nullptr, GMRF_ERR_ALLOC, "context");
    g->N = N;
    g->nnz = (int64_t)col.size();
    g->kappa = kappa;
    g->stream = (cudaStream_t)stream;
    cudaGetDevice(&g->device);
    auto bail = [&](int code) {
        std::snprintf(g_create_err, sizeof(g_create_err), "%s", g->err);
        gmrf_destroy(g);
        return code;
    };
    if (cudaMalloc((void **)&g->rowptr, 4 * (size_t)(N + 1)) != cudaSuccess ||
        cudaMalloc((void **)&g->col, 4 * (size_t)g->nnz) != cudaSuccess ||
        cudaMalloc((void **)&g->val, 8 * (size_t)g->nnz) != cudaSuccess ||
        cudaMalloc((void **)&g->minv, 8 * (size_t)N) != cudaSuccess ||
        cudaMalloc((void **)&g->sqrtc, 8 * (size_t)N) != cudaSuccess ||
        cudaMalloc((void **)&g->n_active, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void **)&g->h_active, sizeof(int)) != cudaSuccess)
        return bail(fail(g, GMRF_ERR_ALLOC, "operator buffers"));
    cudaError_t e = cudaMemcpyAsync(g->rowptr, rowptr.data(), 4 * (size_t)(N + 1), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->col, col.data(), 4 * (size_t)g->nnz, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->val, val.data(), 8 * (size_t)g->nnz, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->minv, minv.data(), 8 * (size_t)N, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->sqrtc, sqrtc.data(), 8 * (size_t)N, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return bail(fail(g, GMRF_ERR_CUDA, "copying the operator: %s", cudaGetErrorString(e)));
    g->info.n_nodes = N;
    g->info.nnz = g->nnz;
    *out = g;
    return GMRF_OK;
}

int gmrf_sample(gmrf_ctx *g, int32_t S, const double *z, double *out, double scale, double mean,
                int32_t lognormal, double rtol, int32_t max_iter) {
    if (!g) return GMRF_ERR_INVALID_ARG;
    if (S < 1 || !z || !out || !(rtol > 0.0 && rtol < 1.0) || max_iter < 1 || !std::isfinite(scale) ||
        !std::isfinite(mean) || (lognormal != 0 && lognormal != 1))
        return fail(g, GMRF_ERR_INVALID_ARG, "S, pointers, rtol in (0, 1), max_iter >= 1, finite scale/mean");
    const int32_t Sp = (S + 1) / 2 * 2;
    int rc = alloc_work(g, Sp);
    if (rc != GMRF_OK) return rc;
    const Geo o = geometry(g->N, Sp);
    const dim3 grid(o.G, o.chunks), block(o.Qt, o.R);
    const size_t sm = sizeof(double2) * o.Qt * o.R;
    const int fin_blocks = (Sp + 7) / 8;
    const double rtol2 = rtol * rtol;
    CKG(cudaMemsetAsync(g->n_active, 0, sizeof(int), g->stream));
    init_kernel<<<grid, block, sm, g->stream>>>(z, S, Sp, g->N, o.tiles, g->sqrtc, g->minv, g->x, g->r,
                                                g->zv, g->p, g->part);
    fin_init_kernel<<<fin_blocks, 256, 0, g->stream>>>(g->part, o.G, Sp, g->scal, g->n_active);
    CKG(cudaGetLastError());
    CKG(cudaMemcpyAsync(g->h_active, g->n_active, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    CKG(cudaStreamSynchronize(g->stream));
    int iters = 0;
    if (g->graph && (g->graph_sp != Sp || g->graph_rtol != rtol)) {
        cudaGraphExecDestroy(g->graph);
        g->graph = nullptr;
    }
    while (*g->h_active > 0 && iters < max_iter) {
        const int k = std::min(kGraphIters, max_iter - iters);
        if (k == kGraphIters) {
            if (!g->graph) {
                cudaStream_t cap;
                CKG(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
                cudaStream_t keep = g->stream;
                g->stream = cap;
                cudaGraph_t gr = nullptr;
                cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
                for (int it = 0; it < kGraphIters && e == cudaSuccess; it++) e = launch_iteration(g, Sp, rtol2);
                cudaError_t e2 = cudaStreamEndCapture(cap, &gr);
                g->stream = keep;
                cudaStreamDestroy(cap);
                if (e == cudaSuccess) e = e2;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&g->graph, gr, 0);
                if (gr) cudaGraphDestroy(gr);
                if (e != cudaSuccess) {
                    g->graph = nullptr;
                    return fail(g, GMRF_ERR_CUDA, "iteration graph: %s", cudaGetErrorString(e));
                }
                g->graph_sp = Sp;
                g->graph_rtol = rtol;
            }
            CKG(cudaGraphLaunch(g->graph, g->stream));
        } else {
            for (int it = 0; it < k; it++) CKG(launch_iteration(g, Sp, rtol2));
        }
        iters += k;
        CKG(cudaMemcpyAsync(g->h_active, g->n_active, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
        CKG(cudaStreamSynchronize(g->stream));
    }
    const int64_t n = (int64_t)g->N * S;
    transform_kernel<<<(unsigned)((n + 255) / 256), 256, 0, g->stream>>>(g->x, g->N, S, Sp, scale, mean,
                                                                         lognormal, out);
    CKG(cudaGetLastError());
    std::vector<double> rel2(Sp);
    CKG(cudaMemcpyAsync(rel2.data(), g->scal + 4 * (size_t)Sp, 8 * (size_t)Sp, cudaMemcpyDeviceToHost, g->stream));
    CKG(cudaStreamSynchronize(g->stream));
    double worst = 0.0;
    for (int32_t s = 0; s < S; s++) worst = std::max(worst, std::sqrt(rel2[s]));
    g->info.iterations = iters;
    g->info.max_relres = worst;
    g->info.last_S = S;
    // per iteration: 12 passes over [N][Sp] binary64 vectors, the matrix (8 + 4 B per entry),
    // row pointers and the diagonal preconditioner
    g->info.bytes_per_iter = 12.0 * 8.0 * (double)g->N * Sp + 12.0 * (double)g->nnz + 12.0 * g->N;
    if (*g->h_active > 0)
        return fail(g, GMRF_ERR_NOT_CONVERGED, "%d samples above rtol after %d iterations (max relres %.3e)",
                    *g->h_active, iters, worst);
    return GMRF_OK;
}

int gmrf_info(const gmrf_ctx *g, gmrf_info_t *info) {
    if (!g || !info) return GMRF_ERR_INVALID_ARG;
    *info = g->info;
    return GMRF_OK;
}

const char *gmrf_last_error(const gmrf_ctx *g) { return g ? g->err : g_create_err; }

void gmrf_destroy(gmrf_ctx *g) {
    if (!g) return;
    if (g->graph) cudaGraphExecDestroy(g->graph);
    void *dev[] = {g->rowptr, g->col, g->val, g->minv, g->sqrtc, g->x, g->r, g->zv, g->p, g->q,
                   g->part, g->scal, g->n_active};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (g->h_active) cudaFreeHost(g->h_active);
    delete g;
}

}  // extern "C"
