// Device Matérn random-field sampler (Section 2.1): x = K^-1 C~^(1/2) z with
// K = kappa^2 C~ + G, all S right-hand sides at once, vectors stored [N][Sp] with the
// sample index innermost (Sp = S rounded up to a multiple of 4; each thread owns one node
// row and two samples, four in the vector update).
//
// GB300 issues binary64 arithmetic at about 1/64 of its binary32 rate, and a binary64 CG
// iteration is bound by that pipe (13 binary64 FMAs per row and sample), so the solve is
// mixed-precision iterative refinement:
//   outer, binary64:  r = b - K x (true residual), stop per sample at ||r|| <= rtol ||b||;
//   inner, binary32:  Jacobi-preconditioned CG on K d = r / ||r|| to a relative tolerance
//                     per sample, a quarter of the reduction still needed to reach rtol,
//                     within [1e-4, 0.1]; then x += ||r|| d.
// A refinement gains up to about four digits (K has condition ~1e3 on the workloads, so
// the binary32 solve is accurate to ~1e-4), the last one only what is left, and the
// final residual is the binary64 one.
// The inner solve takes Chronopoulos and Gear's form of preconditioned CG (one reduction
// per iteration): with z = M^-1 r and w = K z, gamma = r.z and delta = z.w give
// beta = gamma / gamma_prev, alpha = gamma / (delta - beta gamma / alpha_prev), and the
// recurrences p = z + beta p, Kp = w + beta Kp, d += alpha p, r -= alpha Kp; in exact
// arithmetic these are the iterates of standard PCG. One inner iteration is two kernels:
//   cg_matvec  w = (K M^-1) r with partial sums of r.z, z.w, r.r; the block that completes
//              the reduction (a two-level, fixed-order sum through arrival counters) forms
//              alpha, beta, the convergence test and the active count for every sample;
//   cg_update  the four vector recurrences, four samples per thread.
// Every reduction has a fixed shape (a grid fixed per context, fixed trees), so results are
// bitwise reproducible; a converged sample takes alpha = beta = 0 from then on, so
// stopping a few iterations later changes nothing. Inner iterations run as replays of a
// graph.
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
constexpr double kInnerTol = 1e-4;     // smallest inner reduction asked of binary32 CG
constexpr double kInnerMax = 0.1;      // largest inner tolerance
constexpr double kInnerSafety = 0.25;  // inner target against the reduction still needed
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
    float *valz = nullptr, *minv32 = nullptr;  // K M^-1 (binary32, CSR values), M^-1
    // padded-row (ELL) copy of the binary32 K M^-1: ell_w entries per row (8 or 16; 0 when
    // some row is longer), padding entries (own column, value 0)
    int32_t ell_w = 0;
    // blocks of the row kernels: the device's SM count times the fewest blocks of 256
    // threads any of them keeps resident, so each launch is one full wave; fixed per
    // context (and so is every reduction shape)
    int32_t grid = 0;
    int32_t *ell_col = nullptr;
    float *ell_valz = nullptr;
    // work vectors, sized for cap_sp samples
    int32_t cap_sp = 0;
    double *b = nullptr, *x = nullptr, *r = nullptr;       // binary64 [N][Sp]
    // binary32 [N][Sp]: inner solution, residual, direction, K times direction, K M^-1 r
    float *d = nullptr, *ri = nullptr, *p = nullptr, *ap = nullptr, *w = nullptr;
    double *part = nullptr;   // [3][Sp][G]: per-sample partial sums, contiguous over blocks
    double *gpart = nullptr;  // [3][Sp][groups]: sums of kGroup consecutive blocks
    unsigned *ctr = nullptr;  // arrival counters of the groups and the top level
    double *scal = nullptr;  // [kScal][Sp], rows below
    float *scal32 = nullptr; // [2][Sp]: alpha, beta in binary32
    int *n_active = nullptr;
    int *h_active = nullptr;  // pinned
    cudaGraphExec_t graph = nullptr;
    int32_t graph_sp = -1;
    gmrf_info_t info{};
    char err[256] = "";
};

namespace {

// rows of scal
// (kGam: r.z of the last inner iteration, kAlp: its alpha, kTolIn: the square of the
// sample's inner tolerance, kTot..kTot+2: this iteration's totals of r.z, z.w, r.r)
enum { kGam = 0, kBbIn, kActIn, kBb, kRr, kScale, kActOut, kAlp, kTolIn, kTot, kScal = kTot + 3 };
#define SCS(row) scal[(size_t)(row) * Sp + s]

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

Geo geometry(int32_t N, int32_t Sp, int32_t grid, int V = 2) {
    Geo o;
    o.Q = Sp / V;
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

// Inner start: r_i = r / ||r|| (binary32, 0 for converged samples), d = p = K p = 0; the
// samples active in the outer loop start the inner one (state 1: first iteration).
__global__ void inner_init_kernel(const double *__restrict__ r, const double *__restrict__ inv_scale, float *d,
                                  float *ri, float *p, float *ap, double *scal, int32_t N, int32_t Sp,
                                  int64_t tiles) {
    if (blockIdx.x == 0 && threadIdx.y == 0) {
        const int lq = blockIdx.y * blockDim.x + threadIdx.x;
        for (int k = 0; k < 2 && lq < Sp / 2; k++) {
            const int32_t s = 2 * lq + k;
            scal[(size_t)kActIn * Sp + s] = scal[(size_t)kActOut * Sp + s] != 0.0 ? 1.0 : 0.0;
        }
    }
    ROW_LOOP
        const double2 is = ld2(inv_scale + s0);
        const double2 rv = ld2(r + o);
        const float2 rf = make_float2(ens::f64_to_f32_rz(rv.x * is.x), ens::f64_to_f32_rz(rv.y * is.y));
        const float2 zero = make_float2(0.f, 0.f);
        stf2(ri + o, rf);
        stf2(d + o, zero);
        stf2(p + o, zero);
        stf2(ap + o, zero);
    }
}

// Two-level completion of the iteration's reduction. Every block has written its partials
// part[w][s][b] (w < kNQ). A block adds itself to its group's counter (groups of kGroup
// consecutive blockIdx.x, all chunks); the group's last block sums the group's partials
// in block order into gpart[w][s][group] and adds itself to the top counter; the last of
// those returns true, with every group sum visible to it. The last arrivals reset the
// counters, so the next launch starts from zero. No block waits for another. Each sum is
// one thread's, over loads issued together, in a fixed order.
constexpr int kGroup = 16;
constexpr int kNQ = 3;  // r.z, z.w, r.r
constexpr int kMatvecV = 4;  // samples per thread in the product
__device__ __noinline__ bool reduce_arrive(const double *part, double *gpart, unsigned *ctr, int G, int32_t Sp) {
    __shared__ int s_last;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    const int ngroups = (G + kGroup - 1) / kGroup;
    const int grp = blockIdx.x / kGroup;
    const int g0 = grp * kGroup, cnt = min(kGroup, G - g0);
    __threadfence();  // this thread's partials before the arrival
    __syncthreads();
    if (tid == 0) {
        const unsigned expect = (unsigned)cnt * gridDim.y;
        const unsigned prev = atomicAdd(ctr + grp, 1u);
        s_last = prev == expect - 1;
        if (s_last) ctr[grp] = 0;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    for (int pr = tid; pr < kNQ * Sp; pr += nt) {
        const double *src = part + (size_t)pr * G + g0;
        double v[kGroup];
#pragma unroll
        for (int b = 0; b < kGroup; b++) v[b] = b < cnt ? __ldcg(src + b) : 0.0;
        double a = 0.0;
#pragma unroll
        for (int b = 0; b < kGroup; b++) a += v[b];
        gpart[(size_t)pr * ngroups + grp] = a;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned prev = atomicAdd(ctr + ngroups, 1u);
        s_last = prev == (unsigned)ngroups - 1;
        if (s_last) ctr[ngroups] = 0;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    return true;
}

// Sum of src[0..n) in index order, loads issued kGroup at a time.
__device__ __forceinline__ double sum_run(const double *src, int n) {
    double a = 0.0;
    for (int b0 = 0; b0 < n; b0 += kGroup) {
        double v[kGroup];
#pragma unroll
        for (int b = 0; b < kGroup; b++) v[b] = b0 + b < n ? __ldcg(src + b0 + b) : 0.0;
#pragma unroll
        for (int b = 0; b < kGroup; b++) a += v[b];
    }
    return a;
}

// The scalar part of an inner iteration, run by the block that completed the reduction:
// the totals of r.z, z.w, r.r from the group sums (one thread per quantity and sample),
// then, one thread per sample s (state act_s: 0 inactive, 1 first iteration, 2 later ones),
//   convergence: r.r <= tol_s^2 ||r_0||^2 ends the inner solve of s (alpha = beta = 0 from
//   then on, so its d, r stay as they are);
//   beta = gamma / gamma_prev (0 on the first iteration), alpha = gamma / (delta - beta
//   gamma / alpha_prev) (gamma / delta on the first), rounded toward zero to binary32; a
//   non-positive denominator (the binary32 recurrence lost K's definiteness) also ends it;
//   and the number of samples still active goes to *n_active.
// Kept out of line: it runs once per launch, and its binary64 arithmetic would otherwise
// set the register budget of the product loop.
__device__ __noinline__ void finish_iteration(const double *gpart, double *scal, float *alpha32, float *beta32,
                                              int *n_active, int32_t Sp) {
    __shared__ int s_count;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    const int ngroups = (gridDim.x + kGroup - 1) / kGroup;
    if (tid == 0) s_count = 0;
    for (int pr = tid; pr < kNQ * Sp; pr += nt)  // one thread per (quantity, sample)
        scal[(size_t)kTot * Sp + pr] = sum_run(gpart + (size_t)pr * ngroups, ngroups);
    __syncthreads();
    int count = 0;
    for (int32_t s = tid; s < Sp; s += nt) {
        const double gam = SCS(kTot), del = SCS(kTot + 1), rrs = SCS(kTot + 2);
        const double act = SCS(kActIn);
        double alpha = 0.0, beta = 0.0;
        if (act != 0.0) {
            if (act == 1.0) SCS(kBbIn) = rrs;
            bool done = rrs <= SCS(kTolIn) * SCS(kBbIn);
            if (!done) {
                double den = del;
                if (act == 2.0) {
                    beta = ens::f32_to_f64(ens::f64_to_f32_rz(gam / SCS(kGam)));
                    den = del - beta * gam / SCS(kAlp);
                }
                if (gam > 0.0 && den > 0.0) {
                    alpha = ens::f32_to_f64(ens::f64_to_f32_rz(gam / den));
                    SCS(kGam) = gam;
                    SCS(kAlp) = alpha;
                    SCS(kActIn) = 2.0;
                    count++;
                } else {
                    done = true;
                }
            }
            if (done) {
                SCS(kActIn) = 0.0;
                alpha = beta = 0.0;
            }
        }
        alpha32[s] = (float)alpha;  // exact: already binary32 values
        beta32[s] = (float)beta;
    }
    if (count) atomicAdd(&s_count, count);
    __syncthreads();
    if (tid == 0) *n_active = s_count;
}

// Loads and stores of four consecutive binary32 samples (16 bytes aligned).
__device__ __forceinline__ void ldv(const float *p, float (&x)[4]) {
    const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    x[0] = t.x;
    x[1] = t.y;
    x[2] = t.z;
    x[3] = t.w;
}
__device__ __forceinline__ void stv(float *p, const float (&x)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
}

// Inner iteration, part 1: w = (K M^-1) r_i, the product with the column-scaled binary32
// matrix (z = M^-1 r_i never stored), and partials of r.z, z.w and r.r over the block's
// rows (binary32 per thread, binary64 across threads). A thread owns one row and V
// samples; blockDim = (Qt lanes, R rows), grid = (G blocks, lane chunks) as in
// geometry(Sp / V lanes), and block b owns the contiguous row tiles
// [b tiles / G, (b + 1) tiles / G). WP = 8 or 16: padded rows (ELL); the block copies the
// indices and values of up to kStageEntries entries of its rows into shared memory at
// once, so each tile then costs one global round trip (its neighbour rows) instead of
// two. WP = 0: CSR rows, read directly. The block that completes the reduction then
// finishes the iteration (finish_iteration).
constexpr int kStageEntries = 2048;
template <int WP, int V>
__global__ void __launch_bounds__(kThreads, 4) cg_matvec_kernel(
    const int32_t *__restrict__ ell_col, const float *__restrict__ ell_valz, const int32_t *__restrict__ rowptr,
    const int32_t *__restrict__ col, const float *__restrict__ valz, const float *__restrict__ minv,
    const float *__restrict__ ri, float *__restrict__ w, int32_t N, int32_t Sp, int64_t tiles, double *part,
    double *gpart, unsigned *ctr, double *scal, float *alpha32, float *beta32, int *n_active) {
    // dynamic shared memory: the staged rows (int32 indices, then binary32 values,
    // max(kStageEntries, WP R) each), later the block's partial tree
    extern __shared__ double smd[];
    float rz[V], zw[V], rr[V];
#pragma unroll
    for (int k = 0; k < V; k++) rz[k] = zw[k] = rr[k] = 0.f;
    const int R = blockDim.y, Qt = blockDim.x, nt = R * Qt;
    const int y = threadIdx.y, xq = threadIdx.x, tid = y * Qt + xq;
    const int lane = blockIdx.y * Qt + xq;
    const bool lane_ok = lane < Sp / V;
    const int s0 = V * lane;
    const int64_t t0 = (int64_t)blockIdx.x * tiles / gridDim.x;
    const int64_t t1 = (int64_t)(blockIdx.x + 1) * tiles / gridDim.x;
    const int cap = WP > 0 ? max(kStageEntries, WP * R) : 0;
    const int ct = WP > 0 ? max(1, kStageEntries / (WP * R)) : 1;  // tiles per staged chunk
    int32_t *scol = reinterpret_cast<int32_t *>(smd);
    float *sval = reinterpret_cast<float *>(scol + cap);
    for (int64_t tc = t0; tc < t1; tc += ct) {
        const int64_t te = min(tc + (int64_t)ct, t1);
        if constexpr (WP > 0) {
            const int64_t r0 = tc * R, r1 = min(te * R, (int64_t)N);
            const int n4 = (int)((r1 - r0) * WP / 4);
            const int4 *gc = reinterpret_cast<const int4 *>(ell_col + r0 * WP);
            const int4 *gv = reinterpret_cast<const int4 *>(ell_valz + r0 * WP);
            __syncthreads();  // the previous chunk's reads are done
            for (int k = tid; k < n4; k += nt) {
                reinterpret_cast<int4 *>(scol)[k] = __ldg(gc + k);
                reinterpret_cast<int4 *>(sval)[k] = __ldg(gv + k);
            }
            __syncthreads();
        }
        for (int64_t t = tc; t < te; t++) {
            const int64_t i = t * R + y;
            if (i >= N || !lane_ok) continue;
            const size_t o = (size_t)i * Sp + s0;
            float acc[V];
#pragma unroll
            for (int k = 0; k < V; k++) acc[k] = 0.f;
            if constexpr (WP > 0) {
                int32_t cj[WP];
                float aj[WP];
                const int4 *cc = reinterpret_cast<const int4 *>(scol + (i - tc * R) * WP);
                const float4 *vv = reinterpret_cast<const float4 *>(sval + (i - tc * R) * WP);
#pragma unroll
                for (int u = 0; u < WP / 4; u++) {
                    const int4 c = cc[u];
                    const float4 v = vv[u];
                    cj[4 * u] = c.x;
                    cj[4 * u + 1] = c.y;
                    cj[4 * u + 2] = c.z;
                    cj[4 * u + 3] = c.w;
                    aj[4 * u] = v.x;
                    aj[4 * u + 1] = v.y;
                    aj[4 * u + 2] = v.z;
                    aj[4 * u + 3] = v.w;
                }
#pragma unroll
                for (int u = 0; u < WP; u++) {
                    float v[V];
                    ldv(ri + (size_t)cj[u] * Sp + s0, v);
#pragma unroll
                    for (int k = 0; k < V; k++) acc[k] = fmaf(aj[u], v[k], acc[k]);
                }
            } else {
                const int32_t k0 = __ldg(rowptr + i), k1 = __ldg(rowptr + i + 1);
                for (int32_t e = k0; e < k1; e++) {
                    const float a = __ldg(valz + e);
                    float v[V];
                    ldv(ri + (size_t)__ldg(col + e) * Sp + s0, v);
#pragma unroll
                    for (int k = 0; k < V; k++) acc[k] = fmaf(a, v[k], acc[k]);
                }
            }
            stv(w + o, acc);
            float rv[V];
            ldv(ri + o, rv);
            const float m = __ldg(minv + i);
#pragma unroll
            for (int k = 0; k < V; k++) {
                const float zv = m * rv[k];
                rz[k] = fmaf(rv[k], zv, rz[k]);
                zw[k] = fmaf(zv, acc[k], zw[k]);
                rr[k] = fmaf(rv[k], rv[k], rr[k]);
            }
        }
    }
    // per-block sums over the rows: a fixed pairwise tree in binary64, [kNQ][V][threads]
    __syncthreads();  // the staging buffer becomes the tree
#pragma unroll
    for (int k = 0; k < V; k++) {
        smd[(0 * V + k) * nt + tid] = ens::f32_to_f64(rz[k]);
        smd[(1 * V + k) * nt + tid] = ens::f32_to_f64(zw[k]);
        smd[(2 * V + k) * nt + tid] = ens::f32_to_f64(rr[k]);
    }
    __syncthreads();
    int p2 = 1;
    while (p2 < R) p2 <<= 1;
    for (int st = p2 >> 1; st > 0; st >>= 1) {
        if (y < st && y + st < R)
#pragma unroll
            for (int q = 0; q < kNQ * V; q++) smd[q * nt + tid] += smd[q * nt + tid + st * Qt];
        __syncthreads();
    }
    if (y == 0 && lane_ok)
#pragma unroll
        for (int q = 0; q < kNQ; q++)
#pragma unroll
            for (int k = 0; k < V; k++)
                part[((size_t)q * Sp + s0 + k) * gridDim.x + blockIdx.x] = smd[(q * V + k) * nt + xq];
    if (reduce_arrive(part, gpart, ctr, gridDim.x, Sp))
        finish_iteration(gpart, scal, alpha32, beta32, n_active, Sp);
}

// Dynamic shared memory of cg_matvec_kernel<WP, V> for a block of (Qt, R).
size_t matvec_smem(int WP, int V, int Qt, int R) {
    const size_t tree = sizeof(double) * kNQ * V * Qt * R;
    const size_t stage = WP > 0 ? 8 * (size_t)std::max(kStageEntries, WP * R) : 0;
    return std::max(tree, stage);
}

// Inner iteration, part 2, four samples per thread: z = M^-1 r, p = z + beta p,
// Kp = w + beta Kp, d += alpha p, r -= alpha Kp.
__global__ void cg_update_kernel(const float *__restrict__ minv, const float *__restrict__ alpha,
                                 const float *__restrict__ beta, const float *__restrict__ w, float *d, float *ri,
                                 float *p, float *ap, int32_t N, int32_t Sp) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t Q4 = Sp / 4;
    if (t >= (int64_t)N * Q4) return;
    const int32_t s0 = (int32_t)(4 * (t % Q4));
    const float m = __ldg(minv + t / Q4);
    const float4 al = __ldg(reinterpret_cast<const float4 *>(alpha + s0));
    const float4 be = __ldg(reinterpret_cast<const float4 *>(beta + s0));
    float4 *const d4 = reinterpret_cast<float4 *>(d) + t;
    float4 *const r4 = reinterpret_cast<float4 *>(ri) + t;
    float4 *const p4 = reinterpret_cast<float4 *>(p) + t;
    float4 *const a4 = reinterpret_cast<float4 *>(ap) + t;
    const float4 wv = __ldcs(reinterpret_cast<const float4 *>(w) + t);
    float4 rv = *r4, pv = *p4, av = *a4, dv = *d4;
    pv.x = fmaf(be.x, pv.x, m * rv.x);
    pv.y = fmaf(be.y, pv.y, m * rv.y);
    pv.z = fmaf(be.z, pv.z, m * rv.z);
    pv.w = fmaf(be.w, pv.w, m * rv.w);
    av.x = fmaf(be.x, av.x, wv.x);
    av.y = fmaf(be.y, av.y, wv.y);
    av.z = fmaf(be.z, av.z, wv.z);
    av.w = fmaf(be.w, av.w, wv.w);
    dv.x = fmaf(al.x, pv.x, dv.x);
    dv.y = fmaf(al.y, pv.y, dv.y);
    dv.z = fmaf(al.z, pv.z, dv.z);
    dv.w = fmaf(al.w, pv.w, dv.w);
    rv.x = fmaf(-al.x, av.x, rv.x);
    rv.y = fmaf(-al.y, av.y, rv.y);
    rv.z = fmaf(-al.z, av.z, rv.z);
    rv.w = fmaf(-al.w, av.w, rv.w);
    *p4 = pv;
    *a4 = av;
    *d4 = dv;
    *r4 = rv;
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
// while rr > rtol^2 bb; the inner right-hand side is r / ||r||, and the inner solve of an
// active sample stops at a relative residual of tol_s = kInnerSafety rtol sqrt(bb / rr),
// the reduction still needed with a margin, clamped to [kInnerTol, kInnerMax]: the last
// refinement does not go four digits past rtol.
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
        const double need = act ? kInnerSafety * sqrt(rtol2 * bb / rr) : kInnerMax;
        const double tin = fmin(kInnerMax, fmax(kInnerTol, need));
        SC(kTolIn) = tin * tin;
        if (act) atomicAdd(n_active, 1);
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
    void *old[] = {g->b, g->x, g->r, g->d, g->ri, g->p, g->ap, g->w, g->part, g->gpart, g->ctr, g->scal, g->scal32};
    for (void *p : old)
        if (p) cudaFree(p);
    g->b = g->x = g->r = nullptr;
    g->d = g->ri = g->p = g->ap = g->w = nullptr;
    g->part = g->gpart = g->scal = nullptr;
    g->ctr = nullptr;
    g->scal32 = nullptr;
    g->cap_sp = 0;
    const size_t n = (size_t)g->N * Sp;
    double **v64[3] = {&g->b, &g->x, &g->r};
    float **v32[5] = {&g->d, &g->ri, &g->p, &g->ap, &g->w};
    for (double **pp : v64)
        if (cudaMalloc((void **)pp, 8 * n) != cudaSuccess)
            return fail(g, GMRF_ERR_ALLOC, "%zu bytes for a work vector", 8 * n);
    for (float **pp : v32)
        if (cudaMalloc((void **)pp, 4 * n) != cudaSuccess)
            return fail(g, GMRF_ERR_ALLOC, "%zu bytes for a work vector", 4 * n);
    constexpr int kMaxGroups = (kMaxBlocks + kGroup - 1) / kGroup;
    if (cudaMalloc((void **)&g->part, 8 * (size_t)kNQ * kMaxBlocks * Sp) != cudaSuccess ||
        cudaMalloc((void **)&g->gpart, 8 * (size_t)kNQ * kMaxGroups * Sp) != cudaSuccess ||
        cudaMalloc((void **)&g->ctr, sizeof(unsigned) * (kMaxGroups + 1)) != cudaSuccess ||
        cudaMalloc((void **)&g->scal, 8 * (size_t)(kScal + 1) * Sp) != cudaSuccess ||
        cudaMalloc((void **)&g->scal32, 4 * (size_t)2 * Sp) != cudaSuccess)
        return fail(g, GMRF_ERR_ALLOC, "reduction buffers");
    CKG(cudaMemsetAsync(g->ctr, 0, sizeof(unsigned) * (kMaxGroups + 1), g->stream));
    CKG(cudaMemsetAsync(g->scal, 0, 8 * (size_t)(kScal + 1) * Sp, g->stream));
    g->cap_sp = Sp;
    if (g->graph) cudaGraphExecDestroy(g->graph);
    g->graph = nullptr;
    g->graph_sp = -1;
    return GMRF_OK;
}

// One inner (binary32) CG iteration: two launches on g's stream.
cudaError_t launch_iteration(gmrf_ctx *g, int32_t Sp) {
    constexpr int V = kMatvecV;
    const Geo o = geometry(g->N, Sp, g->grid, V);
    const dim3 grid(o.G, o.chunks), block(o.Qt, o.R);
    float *alpha = g->scal32, *beta = g->scal32 + Sp;
#define CG_MATVEC(WP)                                                                                           \
    cg_matvec_kernel<WP, V><<<grid, block, matvec_smem(WP, V, o.Qt, o.R), g->stream>>>(g->ell_col, g->ell_valz, g->rowptr, g->col, g->valz, \
                                                            g->minv32, g->ri, g->w, g->N, Sp, o.tiles, g->part,  \
                                                            g->gpart, g->ctr, g->scal, alpha, beta, g->n_active)
    if (g->ell_w == 8)
        CG_MATVEC(8);
    else if (g->ell_w == 16)
        CG_MATVEC(16);
    else
        CG_MATVEC(0);
#undef CG_MATVEC
    const int64_t n4 = (int64_t)g->N * Sp / 4;
    cg_update_kernel<<<(unsigned)((n4 + 255) / 256), 256, 0, g->stream>>>(g->minv32, alpha, beta, g->w, g->d, g->ri,
                                                                         g->p, g->ap, g->N, Sp);
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
    // the inner iteration multiplies by K M^-1 (M = diag K, the Jacobi preconditioner):
    // entries K_ij / K_jj, formed in binary64 and rounded once
    std::vector<float> minv32(N), valz(val.size());
    std::vector<double> sqrtc(N);
    for (int32_t i = 0; i < N; i++) {
        minv32[i] = (float)(1.0 / diag[i]);
        sqrtc[i] = std::sqrt(cl[i]);
    }
    for (int32_t i = 0; i < N; i++)
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++) valz[k] = (float)(val[k] / diag[col[k]]);
    int32_t wmax = 0;
    for (int32_t i = 0; i < N; i++) wmax = std::max(wmax, rowptr[i + 1] - rowptr[i]);
    const int32_t ell_w = wmax <= 8 ? 8 : (wmax <= 16 ? 16 : 0);
    std::vector<int32_t> ell_col((size_t)N * std::max(ell_w, 1));
    std::vector<float> ell_valz((size_t)N * std::max(ell_w, 1));
    for (int32_t i = 0; ell_w > 0 && i < N; i++)
        for (int32_t u = 0; u < ell_w; u++) {
            const int32_t k = rowptr[i] + u;
            const bool ok = k < rowptr[i + 1];
            ell_col[(size_t)i * ell_w + u] = ok ? col[k] : i;
            ell_valz[(size_t)i * ell_w + u] = ok ? valz[k] : 0.f;
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
        cudaMalloc((void **)&g->valz, 4 * (size_t)g->nnz) != cudaSuccess ||
        cudaMalloc((void **)&g->minv32, 4 * (size_t)N) != cudaSuccess ||
        cudaMalloc((void **)&g->ell_col, 4 * ell_col.size()) != cudaSuccess ||
        cudaMalloc((void **)&g->ell_valz, 4 * ell_valz.size()) != cudaSuccess ||
        cudaMalloc((void **)&g->sqrtc, 8 * (size_t)N) != cudaSuccess ||
        cudaMalloc((void **)&g->n_active, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void **)&g->h_active, sizeof(int)) != cudaSuccess)
        return bail(fail(g, GMRF_ERR_ALLOC, "operator buffers"));
    cudaError_t e = cudaMemcpyAsync(g->rowptr, rowptr.data(), 4 * (size_t)(N + 1), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->col, col.data(), 4 * (size_t)g->nnz, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->val, val.data(), 8 * (size_t)g->nnz, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->valz, valz.data(), 4 * (size_t)g->nnz, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->minv32, minv32.data(), 4 * (size_t)N, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->ell_col, ell_col.data(), 4 * ell_col.size(), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->ell_valz, ell_valz.data(), 4 * ell_valz.size(), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->sqrtc, sqrtc.data(), 8 * (size_t)N, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return bail(fail(g, GMRF_ERR_CUDA, "copying the operator: %s", cudaGetErrorString(e)));
    {
        int sms = 0, per = 0, least = 1 << 20;
        const size_t smb = sizeof(double2) * kThreads;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
        const struct {
            const void *f;
            size_t smem;
        } fns[] = {{(const void *)cg_matvec_kernel<8, kMatvecV>, kNQ * kMatvecV * 8 * kThreads},
                   {(const void *)cg_matvec_kernel<16, kMatvecV>, kNQ * kMatvecV * 8 * kThreads},
                   {(const void *)cg_matvec_kernel<0, kMatvecV>, kNQ * kMatvecV * 8 * kThreads},
                   {(const void *)inner_init_kernel, 0},
                   {(const void *)residual_kernel, smb}, {(const void *)rhs_kernel, smb}};
        for (const auto &k : fns)
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k.f, kThreads, k.smem) == cudaSuccess && per > 0)
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
    const int32_t Sp = (S + 3) / 4 * 4;
    int rc = alloc_work(g, Sp);
    if (rc != GMRF_OK) return rc;
    const Geo o = geometry(g->N, Sp, g->grid);
    const dim3 grid(o.G, o.chunks), block(o.Qt, o.R);
    const size_t sm = sizeof(double2) * o.Qt * o.R;
    double *inv_scale = g->scal + (size_t)kScal * Sp;
    // binary64 right-hand side and residual
    CKG(cudaMemsetAsync(g->n_active, 0, sizeof(int), g->stream));
    rhs_kernel<<<grid, block, sm, g->stream>>>(z, S, Sp, g->N, o.tiles, g->sqrtc, g->b, g->x, g->r, g->part);
    fin_outer_kernel<<<Sp, kFinThreads, 0, g->stream>>>(g->part, o.G, Sp, rtol * rtol, 1, g->scal, inv_scale,
                                                        g->n_active);
    CKG(cudaGetLastError());
    if ((rc = read_active(g)) != GMRF_OK) return rc;
    if (g->graph && g->graph_sp != Sp) {
        cudaGraphExecDestroy(g->graph);
        g->graph = nullptr;
    }
    int iters = 0, refinements = 0;
    while (*g->h_active > 0 && iters < max_iter && refinements < kMaxRefinements) {
        // inner binary32 solve of K d = r / ||r||, started by the samples the outer test
        // left active (their count is in h_active)
        inner_init_kernel<<<grid, block, 0, g->stream>>>(g->r, inv_scale, g->d, g->ri, g->p, g->ap, g->scal, g->N,
                                                         Sp, o.tiles);
        CKG(cudaGetLastError());
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
                    for (int it = 0; it < kGraphIters && e == cudaSuccess; it++) e = launch_iteration(g, Sp);
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
                }
                CKG(cudaGraphLaunch(g->graph, g->stream));
            } else {
                for (int it = 0; it < k; it++) CKG(launch_iteration(g, Sp));
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
    // per inner iteration: 11 passes over binary32 [N][Sp] vectors (r read and w written by
    // the product; r, p, Kp, w, d read and p, Kp, d, r written by the update), the binary32
    // matrix (4 + 4 B per entry) and the binary32 preconditioner
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
    void *dev[] = {g->rowptr, g->col, g->val, g->valz, g->minv32, g->ell_col, g->ell_valz, g->sqrtc, g->b,
                   g->x, g->r, g->d, g->ri, g->p, g->ap, g->w, g->part, g->gpart, g->ctr, g->scal,
                   g->scal32, g->n_active};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (g->h_active) cudaFreeHost(g->h_active);
    delete g;
}

}  // extern "C"
