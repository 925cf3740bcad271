// Device Matérn random-field sampler (Section 2.1): x = K^-1 C~^(1/2) z with
// K = kappa^2 C~ + G, all S right-hand sides at once, vectors stored [N][Sp] with the
// sample index innermost (Sp = S rounded up to even; each thread owns one node row and
// two samples).
//
// GB300 issues binary64 arithmetic at about 1/64 of its binary32 rate, and a binary64 CG
// iteration is bound by that pipe (13 binary64 FMAs per row and sample), so the solve is
// mixed-precision iterative refinement:
//   outer, binary64:  r = b - K x (true residual), stop per sample at ||r|| <= rtol ||b||;
//   inner, binary32:  Jacobi-preconditioned CG on K d = r / ||r|| to relative tolerance
//                     max(rtol, 1e-4), then x += ||r|| d.
// Each refinement gains about four digits (K has condition ~1e3 on the workloads, so the
// binary32 solve is accurate to ~1e-4), and the final residual is the binary64 one.
// One inner iteration is five kernels:
//   spmv_dot   q = K p (binary32 matrix), per-block partial sums of p.q;
//   fin_alpha  alpha_s = rz_s / (p.q)_s (0 once sample s has converged);
//   update     d += alpha p, r -= alpha q, partial sums of r.z and r.r with z = M^-1 r;
//   fin_beta   beta_s, convergence test, active count;
//   pupdate    p = M^-1 r + beta p.
// Every reduction has a fixed shape (a grid fixed per context, fixed trees), so results are bitwise
// reproducible; a converged sample takes alpha = beta = 0 from then on, so stopping a
// few iterations later changes nothing. Inner iterations run as replays of a graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gmrf.h"
#include "ens_bits.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 4096;  // upper bound of the row kernels' grid (see gmrf_ctx::grid)
constexpr int kGraphIters = 8;
constexpr double kInnerTol = 1e-4;
constexpr int kMaxRefinements = 16;

thread_local char g_create_err[256] = "";

}  // namespace

struct gmrf_ctx {
    int32_t N = 0;
    int64_t nnz = 0;
    double kappa = 0.0;
    cudaStream_t stream = nullptr;
    int device = 0;
    int32_t *rowptr = nullptr, *col = nullptr;
    double *val = nullptr, *sqrtc = nullptr;
    float *val32 = nullptr, *minv32 = nullptr;
    // padded-row (ELL) copy of the binary32 matrix: ell_w entries per row (8 or 16; 0 when
    // some row is longer), padding entries (own column, value 0)
    int32_t ell_w = 0;
    // blocks of the row kernels: the device's SM count times the fewest blocks of 256
    // threads any of them keeps resident, so each launch is one full wave; fixed per
    // context (and so is every reduction shape)
    int32_t grid = 0;
    int32_t *ell_col = nullptr;
    float *ell_val = nullptr;
    // work vectors, sized for cap_sp samples
    int32_t cap_sp = 0;
    double *b = nullptr, *x = nullptr, *r = nullptr;       // binary64 [N][Sp]
    float *d = nullptr, *ri = nullptr, *p = nullptr, *q = nullptr;  // binary32 [N][Sp]
    double *part = nullptr;  // [2][Sp][G]: per-sample partial sums, contiguous over blocks
    double *scal = nullptr;  // [kScal][Sp], rows below
    float *scal32 = nullptr; // [2][Sp]: alpha, beta in binary32
    int *n_active = nullptr;
    int *h_active = nullptr;  // pinned
    cudaGraphExec_t graph = nullptr;
    int32_t graph_sp = -1;
    double graph_tol = -1.0;
    gmrf_info_t info{};
    char err[256] = "";
};

namespace {

// rows of scal
enum { kRz = 0, kBbIn, kActIn, kBb, kRr, kScale, kActOut, kScal };

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

Geo geometry(int32_t N, int32_t Sp, int32_t grid) {
    Geo o;
    o.Q = Sp / 2;
    o.Qt = std::min(o.Q, kThreads);
    o.R = std::max(1, kThreads / o.Qt);
    o.tiles = ((int64_t)N + o.R - 1) / o.R;
    o.G = (int)std::min<int64_t>(o.tiles, grid);
    o.chunks = (o.Q + o.Qt - 1) / o.Qt;
    return o;
}

// Sum the per-thread partials of a block over its rows (fixed pairwise tree, binary64)
// and write them to part[w][s][blockIdx.x].
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

// binary32 pair -> binary64 pair on the integer pipe (exact)
__device__ __forceinline__ double2 widen(float2 a) { return make_double2(ens::f32_to_f64(a.x), ens::f32_to_f64(a.y)); }

__device__ __forceinline__ double2 ld2(const double *p) { return *reinterpret_cast<const double2 *>(p); }
__device__ __forceinline__ void st2(double *p, double2 v) { *reinterpret_cast<double2 *>(p) = v; }
__device__ __forceinline__ float2 ldf2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void stf2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }

#define ROW_LOOP                                                          \
    const int lane_q = blockIdx.y * blockDim.x + threadIdx.x;             \
    const bool lane_ok = lane_q < Sp / 2;                                 \
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {             \
        const int64_t i = t * blockDim.y + threadIdx.y;                   \
        if (i >= N || !lane_ok) continue;                                 \
        const int s0 = 2 * lane_q;                                        \
        const size_t o = (size_t)i * Sp + s0;

// b = C~^(1/2) z (padding samples 0), x = 0, r = b; partials of r.r.
__global__ void rhs_kernel(const double *__restrict__ zin, int32_t S, int32_t Sp, int32_t N, int64_t tiles,
                           const double *__restrict__ sqrtc, double *b, double *x, double *r, double *part) {
    extern __shared__ double2 sm[];
    double2 rr = make_double2(0.0, 0.0);
    ROW_LOOP
        const double c = sqrtc[i];
        const double z0 = s0 < S ? zin[i * S + s0] : 0.0;
        const double z1 = s0 + 1 < S ? zin[i * S + s0 + 1] : 0.0;
        const double2 bv = make_double2(c * z0, c * z1);
        st2(b + o, bv);
        st2(r + o, bv);
        st2(x + o, make_double2(0.0, 0.0));
        rr.x = fma(bv.x, bv.x, rr.x);
        rr.y = fma(bv.y, bv.y, rr.y);
    }
    block_partial(rr, sm, part, 0, gridDim.x, Sp, lane_q);
}

// x += scale d (the inner correction, samples still active).
__global__ void correct_kernel(const float *__restrict__ d, const double *__restrict__ scale, double *x,
                               int32_t N, int32_t Sp) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * Sp / 2) return;
    const int32_t s0 = (int32_t)(2 * (t % (Sp / 2)));
    const double2 sc = ld2(scale + s0);
    const double2 dv = widen(ldf2(d + 2 * t));
    double2 xv = ld2(x + 2 * t);
    xv.x = fma(sc.x, dv.x, xv.x);
    xv.y = fma(sc.y, dv.y, xv.y);
    st2(x + 2 * t, xv);
}

// r = b - K x in binary64, partials of r.r.
__global__ void residual_kernel(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                const double *__restrict__ val, const double *__restrict__ x,
                                const double *__restrict__ b, double *r, int32_t N, int32_t Sp, int64_t tiles,
                                double *part) {
    extern __shared__ double2 sm[];
    double2 rr = make_double2(0.0, 0.0);
    ROW_LOOP
        double2 acc = ld2(b + o);
        const int32_t k0 = __ldg(rowptr + i), k1 = __ldg(rowptr + i + 1);
        for (int32_t k = k0; k < k1; k++) {
            const double a = __ldg(val + k);
            const double2 v = __ldg(reinterpret_cast<const double2 *>(x + (size_t)__ldg(col + k) * Sp + s0));
            acc.x = fma(-a, v.x, acc.x);
            acc.y = fma(-a, v.y, acc.y);
        }
        st2(r + o, acc);
        rr.x = fma(acc.x, acc.x, rr.x);
        rr.y = fma(acc.y, acc.y, rr.y);
    }
    block_partial(rr, sm, part, 0, gridDim.x, Sp, lane_q);
}

// Inner start: r_i = r / ||r|| (binary32, 0 for converged samples), d = 0, p = M^-1 r_i;
// partials of r_i.z and r_i.r_i.
__global__ void inner_init_kernel(const double *__restrict__ r, const double *__restrict__ inv_scale,
                                  const float *__restrict__ minv, float *d, float *ri, float *p, int32_t N,
                                  int32_t Sp, int64_t tiles, double *part) {
    extern __shared__ double2 sm[];
    float2 rz = make_float2(0.f, 0.f), rr = rz;
    ROW_LOOP
        const double2 is = ld2(inv_scale + s0);
        const double2 rv = ld2(r + o);
        const float2 rf = make_float2(ens::f64_to_f32_rz(rv.x * is.x), ens::f64_to_f32_rz(rv.y * is.y));
        const float m = minv[i];
        const float2 zz = make_float2(m * rf.x, m * rf.y);
        stf2(ri + o, rf);
        stf2(d + o, make_float2(0.f, 0.f));
        stf2(p + o, zz);
        rz.x = fmaf(rf.x, zz.x, rz.x);
        rz.y = fmaf(rf.y, zz.y, rz.y);
        rr.x = fmaf(rf.x, rf.x, rr.x);
        rr.y = fmaf(rf.y, rf.y, rr.y);
    }
    block_partial(widen(rz), sm, part, 0, gridDim.x, Sp, lane_q);
    block_partial(widen(rr), sm, part, 1, gridDim.x, Sp, lane_q);
}

// q = K p (binary32) and partials of p.q.
__global__ void spmv_dot_kernel(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                const float *__restrict__ val, const float *__restrict__ p,
                                float *__restrict__ q, int32_t N, int32_t Sp, int64_t tiles, double *part) {
    extern __shared__ double2 sm[];
    float2 pq = make_float2(0.f, 0.f);
    ROW_LOOP
        float2 acc = make_float2(0.f, 0.f);
        const int32_t k0 = __ldg(rowptr + i), k1 = __ldg(rowptr + i + 1);
        // the first kUnroll entries: all column indices first, then all vector loads, so a
        // row costs two dependent round trips instead of one per entry
        constexpr int kUnroll = 7;
        int32_t cj[kUnroll];
        float aj[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const bool ok = k0 + u < k1;
            cj[u] = ok ? __ldg(col + k0 + u) : (int32_t)i;
            aj[u] = ok ? __ldg(val + k0 + u) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const float2 v = __ldg(reinterpret_cast<const float2 *>(p + (size_t)cj[u] * Sp + s0));
            acc.x = fmaf(aj[u], v.x, acc.x);
            acc.y = fmaf(aj[u], v.y, acc.y);
        }
        for (int32_t k = k0 + kUnroll; k < k1; k++) {
            const float a = __ldg(val + k);
            const float2 v = __ldg(reinterpret_cast<const float2 *>(p + (size_t)__ldg(col + k) * Sp + s0));
            acc.x = fmaf(a, v.x, acc.x);
            acc.y = fmaf(a, v.y, acc.y);
        }
        stf2(q + o, acc);
        const float2 pv = ldf2(p + o);
        pq.x = fmaf(pv.x, acc.x, pq.x);
        pq.y = fmaf(pv.y, acc.y, pq.y);
    }
    block_partial(widen(pq), sm, part, 0, gridDim.x, Sp, lane_q);
}

// The same product from the padded rows: the column indices and values of a row are
// WP / 4 vector loads that do not wait for the row pointers, so a row costs two dependent
// round trips (indices, then the WP gathers).
template <int WP>
__global__ void spmv_ell_kernel(const int32_t *__restrict__ ell_col, const float *__restrict__ ell_val,
                                const float *__restrict__ p, float *__restrict__ q, int32_t N, int32_t Sp,
                                int64_t tiles, double *part) {
    extern __shared__ double2 sm[];
    float2 pq = make_float2(0.f, 0.f);
    ROW_LOOP
        int32_t cj[WP];
        float aj[WP];
        const int4 *cc = reinterpret_cast<const int4 *>(ell_col + (size_t)i * WP);
        const float4 *vv = reinterpret_cast<const float4 *>(ell_val + (size_t)i * WP);
#pragma unroll
        for (int u = 0; u < WP / 4; u++) {
            const int4 c = __ldg(cc + u);
            const float4 v = __ldg(vv + u);
            cj[4 * u] = c.x;
            cj[4 * u + 1] = c.y;
            cj[4 * u + 2] = c.z;
            cj[4 * u + 3] = c.w;
            aj[4 * u] = v.x;
            aj[4 * u + 1] = v.y;
            aj[4 * u + 2] = v.z;
            aj[4 * u + 3] = v.w;
        }
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < WP; u++) {
            const float2 v = __ldg(reinterpret_cast<const float2 *>(p + (size_t)cj[u] * Sp + s0));
            acc.x = fmaf(aj[u], v.x, acc.x);
            acc.y = fmaf(aj[u], v.y, acc.y);
        }
        stf2(q + o, acc);
        const float2 pv = ldf2(p + o);
        pq.x = fmaf(pv.x, acc.x, pq.x);
        pq.y = fmaf(pv.y, acc.y, pq.y);
    }
    block_partial(widen(pq), sm, part, 0, gridDim.x, Sp, lane_q);
}

// d += alpha p, r -= alpha q; partials of r.z (z = M^-1 r) and r.r.
__global__ void update_kernel(const float *__restrict__ minv, const float *__restrict__ alpha, float *d,
                              float *ri, const float *__restrict__ p, const float *__restrict__ q, int32_t N,
                              int32_t Sp, int64_t tiles, double *part) {
    extern __shared__ double2 sm[];
    float2 rz = make_float2(0.f, 0.f), rr = rz;
    const int lq = blockIdx.y * blockDim.x + threadIdx.x;
    const float2 al = lq < Sp / 2 ? ldf2(alpha + 2 * lq) : make_float2(0.f, 0.f);
    ROW_LOOP
        const float2 pv = ldf2(p + o), qv = ldf2(q + o);
        float2 dv = ldf2(d + o), rv = ldf2(ri + o);
        dv.x = fmaf(al.x, pv.x, dv.x);
        dv.y = fmaf(al.y, pv.y, dv.y);
        rv.x = fmaf(-al.x, qv.x, rv.x);
        rv.y = fmaf(-al.y, qv.y, rv.y);
        stf2(d + o, dv);
        stf2(ri + o, rv);
        const float m = minv[i];
        rz.x = fmaf(rv.x, m * rv.x, rz.x);
        rz.y = fmaf(rv.y, m * rv.y, rz.y);
        rr.x = fmaf(rv.x, rv.x, rr.x);
        rr.y = fmaf(rv.y, rv.y, rr.y);
    }
    block_partial(widen(rz), sm, part, 0, gridDim.x, Sp, lane_q);
    block_partial(widen(rr), sm, part, 1, gridDim.x, Sp, lane_q);
}

// p = M^-1 r + beta p.
__global__ void pupdate_kernel(const float *__restrict__ beta, const float *__restrict__ minv,
                               const float *__restrict__ ri, float *p, int32_t N, int32_t Sp) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * Sp / 2) return;
    const int32_t s0 = (int32_t)(2 * (t % (Sp / 2)));
    const float m = minv[t / (Sp / 2)];
    const float2 b = ldf2(beta + s0);
    const float2 rv = ldf2(ri + 2 * t);
    float2 pv = ldf2(p + 2 * t);
    pv.x = fmaf(b.x, pv.x, m * rv.x);
    pv.y = fmaf(b.y, pv.y, m * rv.y);
    stf2(p + 2 * t, pv);
}

// Sum of part[w][s][0..G) by the block of sample s (blockIdx.x = s): fixed strided
// assignment to the threads, then a fixed pairwise tree.
constexpr int kFinThreads = 128;
__device__ __forceinline__ double block_total(const double *part, int w, int G, int32_t Sp, int s) {
    __shared__ double red[kFinThreads];
    const double *src = part + ((size_t)w * Sp + s) * G;
    double a = 0.0;
    for (int b = threadIdx.x; b < G; b += kFinThreads) a += src[b];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int st = kFinThreads / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    const double t = red[0];
    __syncthreads();
    return t;
}

#define FIN_SAMPLE                            \
    const int s = blockIdx.x;                  \
    const bool lead = threadIdx.x == 0;
#define SC(row) scal[(size_t)(row) * Sp + s]

// Outer test after a residual: rr = ||r||^2 (first: also ||b||^2); a sample stays active
// while rr > rtol^2 bb; the inner right-hand side is r / ||r||.
__global__ void fin_outer_kernel(const double *part, int G, int32_t Sp, double rtol2, int first, double *scal,
                                 double *inv_scale, int *n_active) {
    FIN_SAMPLE
    const double rr = block_total(part, 0, G, Sp, s);
    if (lead) {
        if (first) SC(kBb) = rr;
        const double bb = SC(kBb);
        const bool act = bb > 0.0 && rr > rtol2 * bb && (first || SC(kActOut) != 0.0);
        SC(kRr) = rr;
        SC(kActOut) = act ? 1.0 : 0.0;
        SC(kScale) = act ? sqrt(rr) : 0.0;
        inv_scale[s] = act ? 1.0 / sqrt(rr) : 0.0;
        if (act) atomicAdd(n_active, 1);
    }
}

__global__ void fin_inner_init_kernel(const double *part, int G, int32_t Sp, double *scal, int *n_active) {
    FIN_SAMPLE
    const double rz = block_total(part, 0, G, Sp, s);
    const double bb = block_total(part, 1, G, Sp, s);
    if (lead) {
        const bool act = bb > 0.0;
        SC(kRz) = rz;
        SC(kBbIn) = bb;
        SC(kActIn) = act ? 1.0 : 0.0;
        if (act) atomicAdd(n_active, 1);
    }
}

__global__ void fin_alpha_kernel(const double *part, int G, int32_t Sp, double *scal, float *alpha32,
                                 int *n_active) {
    FIN_SAMPLE
    if (s == 0 && lead) *n_active = 0;
    const double pq = block_total(part, 0, G, Sp, s);
    if (lead) {
        const bool act = SC(kActIn) != 0.0;
        alpha32[s] = (act && pq > 0.0) ? ens::f64_to_f32_rz(SC(kRz) / pq) : 0.f;
    }
}

__global__ void fin_beta_kernel(const double *part, int G, int32_t Sp, double tol2, double *scal, float *beta32,
                                int *n_active) {
    FIN_SAMPLE
    const double rz = block_total(part, 0, G, Sp, s);
    const double rr = block_total(part, 1, G, Sp, s);
    if (lead) {
        float beta = 0.f;
        if (SC(kActIn) != 0.0) {
            const bool done = rr <= tol2 * SC(kBbIn);
            if (!done && SC(kRz) > 0.0) beta = ens::f64_to_f32_rz(rz / SC(kRz));
            SC(kRz) = rz;
            if (done)
                SC(kActIn) = 0.0;
            else
                atomicAdd(n_active, 1);
        }
        beta32[s] = beta;
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
    void *old[] = {g->b, g->x, g->r, g->d, g->ri, g->p, g->q, g->part, g->scal, g->scal32};
    for (void *p : old)
        if (p) cudaFree(p);
    g->b = g->x = g->r = nullptr;
    g->d = g->ri = g->p = g->q = nullptr;
    g->part = g->scal = nullptr;
    g->scal32 = nullptr;
    g->cap_sp = 0;
    const size_t n = (size_t)g->N * Sp;
    double **v64[3] = {&g->b, &g->x, &g->r};
    float **v32[4] = {&g->d, &g->ri, &g->p, &g->q};
    for (double **pp : v64)
        if (cudaMalloc((void **)pp, 8 * n) != cudaSuccess)
            return fail(g, GMRF_ERR_ALLOC, "%zu bytes for a work vector", 8 * n);
    for (float **pp : v32)
        if (cudaMalloc((void **)pp, 4 * n) != cudaSuccess)
            return fail(g, GMRF_ERR_ALLOC, "%zu bytes for a work vector", 4 * n);
    if (cudaMalloc((void **)&g->part, 8 * (size_t)2 * kMaxBlocks * Sp) != cudaSuccess ||
        cudaMalloc((void **)&g->scal, 8 * (size_t)(kScal + 1) * Sp) != cudaSuccess ||
        cudaMalloc((void **)&g->scal32, 4 * (size_t)2 * Sp) != cudaSuccess)
        return fail(g, GMRF_ERR_ALLOC, "reduction buffers");
    g->cap_sp = Sp;
    if (g->graph) cudaGraphExecDestroy(g->graph);
    g->graph = nullptr;
    g->graph_sp = -1;
    return GMRF_OK;
}

// One inner (binary32) CG iteration: five launches on g's stream.
cudaError_t launch_iteration(gmrf_ctx *g, int32_t Sp, double tol2) {
    const Geo o = geometry(g->N, Sp, g->grid);
    const dim3 grid(o.G, o.chunks), block(o.Qt, o.R);
    const size_t sm = sizeof(double2) * o.Qt * o.R;
    float *alpha = g->scal32, *beta = g->scal32 + Sp;
    if (g->ell_w == 8)
        spmv_ell_kernel<8><<<grid, block, sm, g->stream>>>(g->ell_col, g->ell_val, g->p, g->q, g->N, Sp, o.tiles,
                                                           g->part);
    else if (g->ell_w == 16)
        spmv_ell_kernel<16><<<grid, block, sm, g->stream>>>(g->ell_col, g->ell_val, g->p, g->q, g->N, Sp, o.tiles,
                                                            g->part);
    else
        spmv_dot_kernel<<<grid, block, sm, g->stream>>>(g->rowptr, g->col, g->val32, g->p, g->q, g->N, Sp, o.tiles,
                                                        g->part);
    fin_alpha_kernel<<<Sp, kFinThreads, 0, g->stream>>>(g->part, o.G, Sp, g->scal, alpha, g->n_active);
    update_kernel<<<grid, block, sm, g->stream>>>(g->minv32, alpha, g->d, g->ri, g->p, g->q, g->N, Sp, o.tiles,
                                                  g->part);
    fin_beta_kernel<<<Sp, kFinThreads, 0, g->stream>>>(g->part, o.G, Sp, tol2, g->scal, beta, g->n_active);
    const int64_t n2 = (int64_t)g->N * Sp / 2;
    pupdate_kernel<<<(unsigned)((n2 + 255) / 256), 256, 0, g->stream>>>(beta, g->minv32, g->ri, g->p, g->N, Sp);
    return cudaGetLastError();
}

int read_active(gmrf_ctx *g) {
    CKG(cudaMemcpyAsync(g->h_active, g->n_active, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    CKG(cudaStreamSynchronize(g->stream));
    return GMRF_OK;
}

}  // namespace

extern "C" {

int gmrf_create(int32_t n_nodes, int32_t n_elems, const double *xyz, const int32_t *tri,
                double corr_length, void *stream, gmrf_ctx **out) {
    gmrf_ctx *g = nullptr;
    if (!out) return fail(g, GMRF_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    if (n_nodes < 1 || n_elems < 1 || !xyz || !tri)
        return fail(g, GMRF_ERR_INVALID_ARG, "mesh sizes or pointers");
    if (!(corr_length > 0.0) || !std::isfinite(corr_length))
        return fail(g, GMRF_ERR_INVALID_ARG, "correlation length must be finite and > 0");
    // Section 2.1: rho = sqrt(8 nu) / kappa, with nu = 1
    const double kappa = std::sqrt(8.0) / corr_length;
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
    std::vector<float> minv32(N), val32(val.size());
    std::vector<double> sqrtc(N);
    for (int32_t i = 0; i < N; i++) {
        minv32[i] = (float)(1.0 / diag[i]);
        sqrtc[i] = std::sqrt(cl[i]);
    }
    for (size_t k = 0; k < val.size(); k++) val32[k] = (float)val[k];
    int32_t wmax = 0;
    for (int32_t i = 0; i < N; i++) wmax = std::max(wmax, rowptr[i + 1] - rowptr[i]);
    const int32_t ell_w = wmax <= 8 ? 8 : (wmax <= 16 ? 16 : 0);
    std::vector<int32_t> ell_col((size_t)N * std::max(ell_w, 1));
    std::vector<float> ell_val((size_t)N * std::max(ell_w, 1));
    for (int32_t i = 0; ell_w > 0 && i < N; i++)
        for (int32_t u = 0; u < ell_w; u++) {
            const int32_t k = rowptr[i] + u;
            const bool ok = k < rowptr[i + 1];
            ell_col[(size_t)i * ell_w + u] = ok ? col[k] : i;
            ell_val[(size_t)i * ell_w + u] = ok ? val32[k] : 0.f;
        }

    g = new (std::nothrow) gmrf_ctx();
    if (!g) return fail(nullptr, GMRF_ERR_ALLOC, "context");
    g->N = N;
    g->nnz = (int64_t)col.size();
    g->ell_w = ell_w;
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
        cudaMalloc((void **)&g->val32, 4 * (size_t)g->nnz) != cudaSuccess ||
        cudaMalloc((void **)&g->minv32, 4 * (size_t)N) != cudaSuccess ||
        cudaMalloc((void **)&g->ell_col, 4 * ell_col.size()) != cudaSuccess ||
        cudaMalloc((void **)&g->ell_val, 4 * ell_val.size()) != cudaSuccess ||
        cudaMalloc((void **)&g->sqrtc, 8 * (size_t)N) != cudaSuccess ||
        cudaMalloc((void **)&g->n_active, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void **)&g->h_active, sizeof(int)) != cudaSuccess)
        return bail(fail(g, GMRF_ERR_ALLOC, "operator buffers"));
    cudaError_t e = cudaMemcpyAsync(g->rowptr, rowptr.data(), 4 * (size_t)(N + 1), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->col, col.data(), 4 * (size_t)g->nnz, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->val, val.data(), 8 * (size_t)g->nnz, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->val32, val32.data(), 4 * (size_t)g->nnz, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->minv32, minv32.data(), 4 * (size_t)N, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->ell_col, ell_col.data(), 4 * ell_col.size(), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->ell_val, ell_val.data(), 4 * ell_val.size(), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->sqrtc, sqrtc.data(), 8 * (size_t)N, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return bail(fail(g, GMRF_ERR_CUDA, "copying the operator: %s", cudaGetErrorString(e)));
    {
        int sms = 0, per = 0, least = 1 << 20;
        const size_t smb = sizeof(double2) * kThreads;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
        const void *fns[] = {(const void *)spmv_ell_kernel<8>, (const void *)spmv_ell_kernel<16>,
                             (const void *)spmv_dot_kernel, (const void *)update_kernel, (const void *)inner_init_kernel,
                             (const void *)residual_kernel, (const void *)rhs_kernel};
        for (const void *f : fns)
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, kThreads, smb) == cudaSuccess && per > 0)
                least = std::min(least, per);
        if (sms <= 0 || least == (1 << 20)) return bail(fail(g, GMRF_ERR_CUDA, "occupancy query failed"));
        g->grid = std::min(kMaxBlocks, sms * least);
    }
    g->info.n_nodes = N;
    g->info.nnz = g->nnz;
    g->info.kappa = kappa;
    *out = g;
    return GMRF_OK;
}

int gmrf_sample(gmrf_ctx *g, int32_t S, const double *z, double *out, double sigma, double mean,
                int32_t lognormal, double rtol, int32_t max_iter) {
    if (!g) return GMRF_ERR_INVALID_ARG;
    if (S < 1 || !z || !out || !(rtol > 0.0 && rtol < 1.0) || max_iter < 1 || !std::isfinite(sigma) ||
        !std::isfinite(mean) || (lognormal != 0 && lognormal != 1))
        return fail(g, GMRF_ERR_INVALID_ARG, "S, pointers, rtol in (0, 1), max_iter >= 1, finite sigma/mean");
    // marginal variance of x for nu = 1 on a 2-D surface: 1 / (4 pi kappa^2) (Section 2.1,
    // Matern variance Gamma(nu) / (Gamma(nu + d/2) (4 pi)^(d/2) kappa^(2 nu))), so the
    // factor sigma sqrt(4 pi) kappa gives marginal standard deviation sigma
    const double scale = sigma > 0.0 ? sigma * std::sqrt(4.0 * 3.14159265358979323846) * g->info.kappa : 1.0;
    const int32_t Sp = (S + 1) / 2 * 2;
    int rc = alloc_work(g, Sp);
    if (rc != GMRF_OK) return rc;
    const Geo o = geometry(g->N, Sp, g->grid);
    const dim3 grid(o.G, o.chunks), block(o.Qt, o.R);
    const size_t sm = sizeof(double2) * o.Qt * o.R;
    const double tol = std::max(rtol, kInnerTol);
    double *inv_scale = g->scal + (size_t)kScal * Sp;
    // binary64 right-hand side and residual
    CKG(cudaMemsetAsync(g->n_active, 0, sizeof(int), g->stream));
    rhs_kernel<<<grid, block, sm, g->stream>>>(z, S, Sp, g->N, o.tiles, g->sqrtc, g->b, g->x, g->r, g->part);
    fin_outer_kernel<<<Sp, kFinThreads, 0, g->stream>>>(g->part, o.G, Sp, rtol * rtol, 1, g->scal, inv_scale,
                                                        g->n_active);
    CKG(cudaGetLastError());
    if ((rc = read_active(g)) != GMRF_OK) return rc;
    if (g->graph && (g->graph_sp != Sp || g->graph_tol != tol)) {
        cudaGraphExecDestroy(g->graph);
        g->graph = nullptr;
    }
    int iters = 0, refinements = 0;
    while (*g->h_active > 0 && iters < max_iter && refinements < kMaxRefinements) {
        // inner binary32 solve of K d = r / ||r||
        CKG(cudaMemsetAsync(g->n_active, 0, sizeof(int), g->stream));
        inner_init_kernel<<<grid, block, sm, g->stream>>>(g->r, inv_scale, g->minv32, g->d, g->ri, g->p, g->N, Sp,
                                                          o.tiles, g->part);
        fin_inner_init_kernel<<<Sp, kFinThreads, 0, g->stream>>>(g->part, o.G, Sp, g->scal, g->n_active);
        CKG(cudaGetLastError());
        if ((rc = read_active(g)) != GMRF_OK) return rc;
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
                    for (int it = 0; it < kGraphIters && e == cudaSuccess; it++) e = launch_iteration(g, Sp, tol * tol);
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
                    g->graph_tol = tol;
                }
                CKG(cudaGraphLaunch(g->graph, g->stream));
            } else {
                for (int it = 0; it < k; it++) CKG(launch_iteration(g, Sp, tol * tol));
            }
            iters += k;
            if ((rc = read_active(g)) != GMRF_OK) return rc;
        }
        // binary64 correction and true residual
        const int64_t n2 = (int64_t)g->N * Sp / 2;
        correct_kernel<<<(unsigned)((n2 + 255) / 256), 256, 0, g->stream>>>(g->d, g->scal + (size_t)kScale * Sp, g->x,
                                                                           g->N, Sp);
        residual_kernel<<<grid, block, sm, g->stream>>>(g->rowptr, g->col, g->val, g->x, g->b, g->r, g->N, Sp,
                                                        o.tiles, g->part);
        CKG(cudaMemsetAsync(g->n_active, 0, sizeof(int), g->stream));
        fin_outer_kernel<<<Sp, kFinThreads, 0, g->stream>>>(g->part, o.G, Sp, rtol * rtol, 0, g->scal, inv_scale,
                                                            g->n_active);
        CKG(cudaGetLastError());
        refinements++;
        if ((rc = read_active(g)) != GMRF_OK) return rc;
    }
    const int64_t n = (int64_t)g->N * S;
    transform_kernel<<<(unsigned)((n + 255) / 256), 256, 0, g->stream>>>(g->x, g->N, S, Sp, scale, mean,
                                                                         lognormal, out);
    CKG(cudaGetLastError());
    std::vector<double> rr(Sp), bb(Sp);
    CKG(cudaMemcpyAsync(rr.data(), g->scal + (size_t)kRr * Sp, 8 * (size_t)Sp, cudaMemcpyDeviceToHost, g->stream));
    CKG(cudaMemcpyAsync(bb.data(), g->scal + (size_t)kBb * Sp, 8 * (size_t)Sp, cudaMemcpyDeviceToHost, g->stream));
    CKG(cudaStreamSynchronize(g->stream));
    double worst = 0.0;
    for (int32_t s = 0; s < S; s++)
        if (bb[s] > 0.0) worst = std::max(worst, std::sqrt(rr[s] / bb[s]));
    g->info.iterations = iters;
    g->info.refinements = refinements;
    g->info.max_relres = worst;
    g->info.last_S = S;
    // per inner iteration: 11 passes over binary32 [N][Sp] vectors, the binary32 matrix
    // (4 + 4 B per entry), row pointers and the binary32 preconditioner
    g->info.bytes_per_iter = 11.0 * 4.0 * (double)g->N * Sp + 8.0 * (double)g->nnz + 8.0 * g->N;  // stored entries only
    // per refinement: correction (x, d) and residual (x gathered, b, r) in binary64
    g->info.bytes_per_refinement = (8.0 * 2 + 4.0 + 8.0 * 3) * (double)g->N * Sp + 12.0 * (double)g->nnz;
    if (*g->h_active > 0)
        return fail(g, GMRF_ERR_NOT_CONVERGED, "%d samples above rtol after %d iterations, %d refinements "
                    "(max relres %.3e)", *g->h_active, iters, refinements, worst);
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
    void *dev[] = {g->rowptr, g->col, g->val, g->val32, g->minv32, g->ell_col, g->ell_val, g->sqrtc, g->b, g->x, g->r, g->d, g->ri,
                   g->p, g->q, g->part, g->scal, g->scal32, g->n_active};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (g->h_active) cudaFreeHost(g->h_active);
    delete g;
}

}  // extern "C"
