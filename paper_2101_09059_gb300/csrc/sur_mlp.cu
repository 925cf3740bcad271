// Surrogate network on the GPU: a GELU multilayer perceptron (n_in -> H -> H -> n_out)
// trained with mean-squared error and Adam, every step in this file's kernels.
//
// Matrix products run on the fifth-generation tensor cores in BF16 with FP32 accumulation
// (tcgen05.mma, the accumulator in tensor memory); master weights, activations, gradients
// and optimiser state stay FP32.
// One training epoch (gather of each shuffled mini-batch, forward, loss, backward, Adam)
// is captured once in a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/sur.h"
#include "ens_bits.cuh"

namespace {

// ---- tensor-core product (tcgen05) ----------------------------------------------------
// One CTA of 128 threads computes a 128 x 32 tile of C (the network's products are a few
// tiles wide, so narrow tiles give more CTAs). Per K stage of 64 the threads stage
// the FP32 operands as BF16 into shared memory in the canonical K-major layout without
// swizzle: 8 x 16-byte core matrices (8 rows of 8 consecutive k), the eight k-groups of a
// row group 128 bytes apart (leading byte offset) and row groups 1024 bytes apart (stride
// byte offset). One thread then issues four tcgen05.mma (M = 128, N = 32, K = 16) into the
// CTA's 32 tensor-memory columns and commits them to an mbarrier that every thread waits
// on (bounded) before the stage is overwritten. At the end warp w reads rows 32w .. 32w+31
// of the accumulator with tcgen05.ld and applies the epilogue.
constexpr int TM = 128, TN = 32, TK = 64;
constexpr int kThreads = 128;
constexpr uint32_t kTmemCols = 32;
constexpr uint32_t kCoreK = 128;                    // bytes between core matrices along k
constexpr uint32_t kCoreMN = (uint32_t)TK * 16u;    // bytes between 8-row groups
constexpr uint32_t kAsBytes = TM / 8 * kCoreMN, kBsBytes = TN / 8 * kCoreMN;
// dynamic shared memory per CTA: at most 8 CTAs fit on an SM, so their 8 x 32 columns
// never exceed the SM's 512 columns of tensor memory and tcgen05.alloc never waits
constexpr uint32_t kTcSmem = 28 * 1024;
constexpr uint32_t kTcWait = 1u << 22;

enum Epi : int {
    kStore = 0,      // C = acc
    kBiasStore = 1,  // C = acc + bias[n]
    kBiasGelu = 2,   // Z = acc + bias[n]; C = gelu(Z) (Z kept for the backward pass)
    kGeluGrad = 3,   // C = acc * gelu'(Z[m][n])
};

// Set when a bounded wait for the tensor cores gave up (read back by the host calls).
__device__ int g_tc_fault;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
           z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Shared-memory matrix descriptor: start address, leading and stride byte offsets (all
// >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(const void *p, uint32_t lbo, uint32_t sbo) {
    const uint32_t a = ens::smem_addr(p);
    return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major,
// N = TN, M = TM.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's row.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
}

// byte offset of element (row r, k) inside a staged operand tile
__device__ __forceinline__ uint32_t core_off(int r, int k) {
    return (uint32_t)(r >> 3) * kCoreMN + (uint32_t)(k >> 3) * kCoreK + (uint32_t)(r & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// One K stage of an operand tile (ROWS rows x TK k) held in registers as 16-byte vectors
// (VR = ROWS * TK / (4 kThreads) per thread). Layout 1: k contiguous in memory (row stride
// sr, a multiple of 4), the vector runs along k; layout 2: rows contiguous (k stride sk, a
// multiple of 4), the vector runs along the rows. Rows beyond R and k beyond K (both
// multiples of 4 in these layouts) read as zero.
template <int ROWS>
struct VecStage {
    static constexpr int VR = ROWS * TK / (4 * kThreads);
    float4 v[VR];
    __device__ __forceinline__ void load(const float *__restrict__ src, int layout, long long sr, long long sk, int r0,
                                         int R, int k0, int K, int tid) {
#pragma unroll
        for (int j = 0; j < VR; j++) {
            const int q = tid + j * kThreads;
            int rr, kk;
            if (layout == 1) {
                rr = q / (TK / 4);
                kk = (q - rr * (TK / 4)) * 4;
            } else {
                kk = q / (ROWS / 4);
                rr = (q - kk * (ROWS / 4)) * 4;
            }
            const int r = r0 + rr, k = k0 + kk;
            v[j] = (r < R && k < K) ? __ldg(reinterpret_cast<const float4 *>(src + (long long)r * sr + (long long)k * sk))
                                    : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    }
    __device__ __forceinline__ void store(unsigned char *dst, int layout, int tid) const {
#pragma unroll
        for (int j = 0; j < VR; j++) {
            const int q = tid + j * kThreads;
            const float x[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
            if (layout == 1) {
                const int rr = q / (TK / 4), kk = (q - rr * (TK / 4)) * 4;
                __nv_bfloat16 h[4];
#pragma unroll
                for (int t = 0; t < 4; t++) h[t] = __float2bfloat16_rn(x[t]);
                // four consecutive k of one row: 8 contiguous bytes of a core matrix
                *reinterpret_cast<uint2 *>(dst + core_off(rr, kk)) = *reinterpret_cast<const uint2 *>(h);
            } else {
                const int kk = q / (ROWS / 4), rr = (q - kk * (ROWS / 4)) * 4;
#pragma unroll
                for (int t = 0; t < 4; t++)
                    *reinterpret_cast<__nv_bfloat16 *>(dst + core_off(rr + t, kk)) = __float2bfloat16_rn(x[t]);
            }
        }
    }
};

// Vector layout of an operand with element (r, k) at src[r sr + k sk]: 1 or 2 as in
// VecStage, 0 for the scalar path.
__device__ __forceinline__ int vec_layout(const float *src, long long sr, long long sk, int R, int K) {
    if ((reinterpret_cast<uintptr_t>(src) & 15u) != 0) return 0;
    if (sk == 1 && (sr & 3) == 0 && (K & 3) == 0) return 1;
    if (sr == 1 && (sk & 3) == 0 && (R & 3) == 0) return 2;
    return 0;
}

// C[M][N] (row stride ldc) = epilogue( sum_k A(m, k) B(k, n) ), FP32 sources staged to BF16.
// A(m, k) = A[m * sam + k * sak], B(k, n) = B[k * sbk + n * sbn]. Out-of-range elements
// are read as zero and not written.
template <int EPI>
__global__ void __launch_bounds__(kThreads) gemm_kernel(int M, int N, int K, const float *__restrict__ A,
                                                        long long sam, long long sak,
                                                        const float *__restrict__ B, long long sbk,
                                                        long long sbn, float *__restrict__ C, int ldc,
                                                        const float *__restrict__ bias,
                                                        float *__restrict__ Z) {
    extern __shared__ __align__(128) unsigned char tsm[];
    unsigned char *As = tsm, *Bs = tsm + kAsBytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(tsm + kAsBytes + kBsBytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(tsm + kAsBytes + kBsBytes + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(ens::smem_addr(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        ens::mbar_init(bar, 1);
        ens::fence_barrier_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    bool ok = true;
    uint32_t phase = 0;
    const int la = vec_layout(A, sam, sak, M, K), lb = vec_layout(B, sbn, sbk, N, K);
    if (la != 0 && lb != 0) {
        // vector path: a stage's loads are issued together, and the next stage's while the
        // tensor cores work on the current one
        VecStage<TM> va;
        VecStage<TN> vb;
        va.load(A, la, sam, sak, m0, M, 0, K, tid);
        vb.load(B, lb, sbn, sbk, n0, N, 0, K, tid);
        for (int k0 = 0; k0 < K && ok; k0 += TK) {
            va.store(As, la, tid);
            vb.store(Bs, lb, tid);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
#pragma unroll
                for (int ks = 0; ks < TK / 16; ks++) {
                    const uint64_t ad = smem_desc(As + ks * 2 * kCoreK, kCoreK, kCoreMN);
                    const uint64_t bd = smem_desc(Bs + ks * 2 * kCoreK, kCoreK, kCoreMN);
                    const uint32_t acc = (k0 > 0 || ks > 0) ? 1u : 0u;
                    asm volatile(
                        "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 ens::smem_addr(bar))
                             : "memory");
            }
            if (k0 + TK < K) {
                va.load(A, la, sam, sak, m0, M, k0 + TK, K, tid);
                vb.load(B, lb, sbn, sbk, n0, N, k0 + TK, K, tid);
            }
            ok = ens::mbar_wait(bar, phase, kTcWait);
            phase ^= 1u;
            tc_fence_after();
            ok = __syncthreads_and(ok);
        }
    }
    for (int k0 = 0; k0 < K && ok && (la == 0 || lb == 0); k0 += TK) {
        // loads in groups of 8 (issued together), then their conversions and shared stores
        constexpr int kA = TM * TK / kThreads, kB = TN * TK / kThreads, kG = 8;
#pragma unroll 1
        for (int j0 = 0; j0 < kA; j0 += kG) {
            float v[kG];
#pragma unroll
            for (int j = 0; j < kG; j++) {
                const int e = tid + (j0 + j) * kThreads;
                const int mm = sak == 1 ? e / TK : e % TM, kk = sak == 1 ? e % TK : e / TM;
                const int m = m0 + mm, k = k0 + kk;
                v[j] = (m < M && k < K) ? __ldg(A + (long long)m * sam + (long long)k * sak) : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < kG; j++) {
                const int e = tid + (j0 + j) * kThreads;
                const int mm = sak == 1 ? e / TK : e % TM, kk = sak == 1 ? e % TK : e / TM;
                *reinterpret_cast<__nv_bfloat16 *>(As + core_off(mm, kk)) = __float2bfloat16_rn(v[j]);
            }
        }
        {
            float v[kB];
#pragma unroll
            for (int j = 0; j < kB; j++) {
                const int e = tid + j * kThreads;
                const int nn = sbk == 1 ? e / TK : e % TN, kk = sbk == 1 ? e % TK : e / TN;
                const int n = n0 + nn, k = k0 + kk;
                v[j] = (n < N && k < K) ? __ldg(B + (long long)k * sbk + (long long)n * sbn) : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < kB; j++) {
                const int e = tid + j * kThreads;
                const int nn = sbk == 1 ? e / TK : e % TN, kk = sbk == 1 ? e % TK : e / TN;
                *reinterpret_cast<__nv_bfloat16 *>(Bs + core_off(nn, kk)) = __float2bfloat16_rn(v[j]);
            }
        }
        // the stores above are generic-proxy writes the tensor core reads through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < TK / 16; ks++) {
                const uint64_t ad = smem_desc(As + ks * 2 * kCoreK, kCoreK, kCoreMN);
                const uint64_t bd = smem_desc(Bs + ks * 2 * kCoreK, kCoreK, kCoreMN);
                const uint32_t acc = (k0 > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             ens::smem_addr(bar))
                         : "memory");
        }
        ok = ens::mbar_wait(bar, phase, kTcWait);
        phase ^= 1u;
        tc_fence_after();
        ok = __syncthreads_and(ok);
    }
    if (!ok) {
        // report, give the products in flight one more bounded wait, then free the columns
        if (tid == 0) atomicExch(&g_tc_fault, 1);
        ens::mbar_wait(bar, phase ^ 1u, kTcWait);
    } else {
        const int m = m0 + 32 * warp + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
        for (int c = 0; c < TN; c += 16) {
            float v[16];
            if (K > 0) {
                tc_ld16(trow + (uint32_t)c, v);
            } else {
#pragma unroll
                for (int j = 0; j < 16; j++) v[j] = 0.0f;
            }
            if (m < M) {
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int n = n0 + c + j;
                    if (n >= N) continue;
                    float x = v[j];
                    const long long o = (long long)m * ldc + n;
                    if constexpr (EPI == kBiasStore) x += bias[n];
                    if constexpr (EPI == kBiasGelu) {
                        x += bias[n];
                        Z[o] = x;
                        x = gelu(x);
                    }
                    if constexpr (EPI == kGeluGrad) x *= gelu_grad(Z[o]);
                    C[o] = x;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// loss = sum (y - t)^2 / count (one block, fixed order); dy = 2 (y - t) / count; with db,
// also the output layer's bias gradient db[n] = sum_m dy[m][n] (rows of `cols` values), in
// the order of colsum_kernel.
__global__ void mse_kernel(const float *__restrict__ y, const float *__restrict__ tgt, long long count,
                           float *__restrict__ dy, float *__restrict__ loss_out, int cols = 0,
                           float *__restrict__ db = nullptr) {
    __shared__ double part[256];
    double s = 0.0;
    const float scale = 2.0f / (float)count;
    for (long long i = threadIdx.x; i < count; i += blockDim.x) {
        const float d = y[i] - tgt[i];
        if (dy) dy[i] = scale * d;
        s += (double)d * (double)d;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss_out) *loss_out = (float)(part[0] / (double)count);
    if (db && dy) {  // dy of this block is visible after the barriers above
        const long long rows = count / cols;
        for (int n = threadIdx.x; n < cols; n += blockDim.x) {
            float t = 0.0f;
            for (long long m = 0; m < rows; m++) t += dy[m * cols + n];
            db[n] = t;
        }
    }
}

// db[n] = sum_m dz[m][n] (one thread per column, fixed order).
__global__ void colsum_kernel(const float *__restrict__ dz, int M, int N, float *__restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.0f;
    for (int m = 0; m < M; m++) s += dz[(long long)m * N + n];
    db[n] = s;
}

// rows of a mini-batch: dst[i][:] = src[perm[off + i]][:]
__global__ void gather_rows_kernel(const float *__restrict__ src, const int *__restrict__ perm, int off,
                                   int rows, int cols, float *__restrict__ dst) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)rows * cols) return;
    const int i = (int)(e / cols), c = (int)(e % cols);
    dst[e] = src[(long long)perm[off + i] * cols + c];
}

// One training step's inputs and targets gathered together (rows * (ca + cb) threads), and
// the Adam step counter advanced for the update that ends the step.
__global__ void gather_step_kernel(const float *__restrict__ A, const float *__restrict__ B, const int *__restrict__ perm,
                                   int off, int rows, int ca, int cb, float *__restrict__ da, float *__restrict__ db,
                                   int *tstep) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e == 0) *tstep += 1;
    const long long na = (long long)rows * ca;
    if (e < na) {
        const int i = (int)(e / ca), c = (int)(e % ca);
        da[e] = A[(long long)perm[off + i] * ca + c];
    } else if (e < na + (long long)rows * cb) {
        const long long f = e - na;
        const int i = (int)(f / cb), c = (int)(f % cb);
        db[f] = B[(long long)perm[off + i] * cb + c];
    }
}

__global__ void tick_kernel(int *t) { *t += 1; }

// Adam (bias-corrected): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), t = *tstep (already advanced).
// Each block forms the bias corrections once, in binary64 from the same binary32 betas the
// moment recurrences use: in binary32 the subtraction 1 - b2^t cancels (b2 = 0.999 leaves
// about 3e-3 at t = 3) and its rounding error of the power becomes a relative error of
// about 1e-5 in the second moment.
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long n, const int *__restrict__ tstep, float lr,
                            float b1, float b2, float eps) {
    __shared__ float corr[2];
    if (threadIdx.x == 0) {
        const double t = (double)*tstep;
        corr[0] = (float)(1.0 - pow((double)b1, t));
        corr[1] = (float)(1.0 - pow((double)b2, t));
    }
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float c1 = corr[0], c2 = corr[1];
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Euclidean norm of every input row x [B][n] in binary64 (one warp per row, fixed
// shuffle tree); with radius >= 0 also flags[b] = 1 where the norm is <= radius.
__global__ void row_norm_kernel(const float *__restrict__ x, long long B, int n, double *__restrict__ norm,
                                double radius, int *__restrict__ flags) {
    const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (row >= B) return;
    double s = 0.0;
    for (int k = lane; k < n; k += 32) {
        const double v = (double)x[row * n + k];
        s = fma(v, v, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const double r = sqrt(s);
        if (norm) norm[row] = r;
        if (flags) flags[row] = r <= radius ? 1 : 0;
    }
}

// u[b][d] = mean[d] + sum_r c[b][r] phi[d][r]  (POD reconstruction, FP32)
__global__ void reconstruct_kernel(const float *__restrict__ c, const float *__restrict__ mean,
                                   const float *__restrict__ phi, int B, long long D, int r,
                                   float *__restrict__ u) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)B * D) return;
    const int b = (int)(e / D);
    const long long d = e % D;
    float s = mean[d];
    for (int k = 0; k < r; k++) s = fmaf(c[(long long)b * r + k], phi[d * r + k], s);
    u[e] = s;
}

// Mean of each coefficient column: mu[i] = sum_m c[m][i] / M (one thread per column).
__global__ void coef_mean_kernel(const float *__restrict__ c, int M, int r, float *__restrict__ mu) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= r) return;
    double s = 0.0;
    for (int m = 0; m < M; m++) s += c[(long long)m * r + i];
    mu[i] = (float)(s / M);
}

// Sample covariance of the coefficients, C[i][j] = sum_m (c_i - mu_i)(c_j - mu_j) / (M - 1).
__global__ void coef_cov_kernel(const float *__restrict__ c, int M, int r, const float *__restrict__ mu,
                                float *__restrict__ C) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= r * r) return;
    const int i = e / r, j = e % r;
    double s = 0.0;
    for (int m = 0; m < M; m++)
        s += ((double)c[(long long)m * r + i] - mu[i]) * ((double)c[(long long)m * r + j] - mu[j]);
    C[e] = M > 1 ? (float)(s / (M - 1)) : 0.0f;
}

// Field statistics implied by the coefficient statistics: mean[d] = u0[d] + phi[d] . mu,
// std[d] = sqrt(phi[d]^T C phi[d]).
__global__ void field_stats_kernel(const float *__restrict__ u0, const float *__restrict__ phi, long long D,
                                   int r, const float *__restrict__ mu, const float *__restrict__ C,
                                   float *__restrict__ mean, float *__restrict__ stdv) {
    extern __shared__ float sh[];  // mu [r], C [r][r]
    for (int e = threadIdx.x; e < r + r * r; e += blockDim.x) sh[e] = e < r ? mu[e] : C[e - r];
    __syncthreads();
    const long long d = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= D) return;
    const float *p = phi + d * r;
    float m = u0[d], v = 0.0f;
    for (int i = 0; i < r; i++) {
        const float pi = p[i];
        m = fmaf(pi, sh[i], m);
        float t = 0.0f;
        for (int j = 0; j < r; j++) t = fmaf(sh[r + i * r + j], p[j], t);
        v = fmaf(pi, t, v);
    }
    mean[d] = m;
    stdv[d] = sqrtf(fmaxf(v, 0.0f));
}

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

long long float_bits(float f) {
    int32_t i;
    memcpy(&i, &f, sizeof(i));
    return i;
}

// The products' dynamic shared memory is above the 48 KB default only in principle (28
// KB), but setting it explicitly once, outside any graph capture, keeps every launch valid.
cudaError_t gemm_setup() {
    cudaError_t e = cudaFuncSetAttribute(gemm_kernel<kStore>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gemm_kernel<kBiasStore>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gemm_kernel<kBiasGelu>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gemm_kernel<kGeluGrad>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    return e;
}

// A bounded tensor-core wait that gave up since the last check (the flag is cleared).
bool tc_faulted() {
    int f = 0;
    if (cudaMemcpyFromSymbol(&f, g_tc_fault, sizeof(int)) != cudaSuccess) return true;
    if (f) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_tc_fault, &zero, sizeof(int));
    }
    return f != 0;
}

template <int EPI>
cudaError_t gemm(cudaStream_t s, int M, int N, int K, const float *A, long long sam, long long sak,
                 const float *B, long long sbk, long long sbn, float *C, int ldc,
                 const float *bias = nullptr, float *Z = nullptr) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid(cdiv(N, TN), cdiv(M, TM));
    gemm_kernel<EPI><<<grid, kThreads, kTcSmem, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, Z);
    return cudaGetLastError();
}

}  // namespace

struct sur_ctx {
    int nin = 0, H = 0, nout = 0, max_batch = 0;
    long long np = 0;  // parameter count
    long long off[6] = {0, 0, 0, 0, 0, 0};  // W1 b1 W2 b2 W3 b3 in the flat vectors
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // private stream for graph capture
    // the backward pass runs its weight gradients on a side branch (fork and join by events)
    cudaStream_t side = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    std::string err;
    float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    // device buffers
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    float *z1 = nullptr, *a1 = nullptr, *z2 = nullptr, *a2 = nullptr, *y = nullptr;
    float *dy = nullptr, *d2 = nullptr, *d1 = nullptr;
    float *xb = nullptr, *tb = nullptr, *loss = nullptr;
    double trust_radius = -1.0;  // inputs with a larger norm are not trusted (sur_fit_trust)
    int *tstep = nullptr, *perm = nullptr;
    long long perm_n = 0;
    float *loss_hist = nullptr;
    long long loss_hist_n = 0;
    cudaGraphExec_t epoch_graph = nullptr;
    long long graph_key[5] = {0, 0, 0, 0, 0};
    std::vector<void *> bufs;
};

namespace {

int sfail(sur_ctx *c, int code, const char *fmt, ...) {
    if (c) {
        char buf[400];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

#define SCK(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return sfail(c, SUR_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
int salloc(sur_ctx *c, T **p, long long n) {
    void *q = nullptr;
    if (cudaMalloc(&q, sizeof(T) * (size_t)(n > 0 ? n : 1)) != cudaSuccess) {
        cudaGetLastError();
        return sfail(c, SUR_ERR_ALLOC, "cudaMalloc of %lld elements", n);
    }
    c->bufs.push_back(q);
    *p = (T *)q;
    return SUR_OK;
}

// Forward pass of B rows already in x (device): z1, a1, z2, a2, y.
int forward(sur_ctx *c, cudaStream_t s, const float *x, int B) {
    const float *W1 = c->p + c->off[0], *b1 = c->p + c->off[1], *W2 = c->p + c->off[2];
    const float *b2 = c->p + c->off[3], *W3 = c->p + c->off[4], *b3 = c->p + c->off[5];
    const int H = c->H;
    SCK((gemm<kBiasGelu>(s, B, H, c->nin, x, c->nin, 1, W1, 1, c->nin, c->a1, H, b1, c->z1)));
    SCK((gemm<kBiasGelu>(s, B, H, H, c->a1, H, 1, W2, 1, H, c->a2, H, b2, c->z2)));
    SCK((gemm<kBiasStore>(s, B, c->nout, H, c->a2, H, 1, W3, 1, H, c->y, c->nout, b3)));
    return SUR_OK;
}

// Loss and gradients of B rows (x, t on device) into c->g; loss to *loss_dev. The chain
// of activation gradients (d2, d1) stays on s; the weight gradients and bias sums that
// branch off it run on c->side, forked and joined by events, so a captured graph holds
// them as parallel branches. Every gradient is written when s continues after the call.
int backward(sur_ctx *c, cudaStream_t s, const float *x, const float *t, int B, float *loss_dev) {
    const int H = c->H, no = c->nout, ni = c->nin;
    const float *W2 = c->p + c->off[2], *W3 = c->p + c->off[4];
    float *gW1 = c->g + c->off[0], *gb1 = c->g + c->off[1], *gW2 = c->g + c->off[2];
    float *gb2 = c->g + c->off[3], *gW3 = c->g + c->off[4], *gb3 = c->g + c->off[5];
    int rc = forward(c, s, x, B);
    if (rc != SUR_OK) return rc;
    mse_kernel<<<1, 256, 0, s>>>(c->y, t, (long long)B * no, c->dy, loss_dev, no, gb3);  // and db3
    SCK(cudaGetLastError());
    // layer 3: dW3 = dy^T a2 (side), db3 = colsum dy (above), d2 = (dy W3) * gelu'(z2)
    SCK(cudaEventRecord(c->ev[0], s));
    SCK(cudaStreamWaitEvent(c->side, c->ev[0], 0));
    SCK((gemm<kStore>(c->side, no, H, B, c->dy, 1, no, c->a2, H, 1, gW3, H)));
    SCK((gemm<kGeluGrad>(s, B, H, no, c->dy, no, 1, W3, H, 1, c->d2, H, nullptr, c->z2)));
    // layer 2: dW2 = d2^T a1 and db2 (side), d1 = (d2 W2) * gelu'(z1)
    SCK(cudaEventRecord(c->ev[1], s));
    SCK(cudaStreamWaitEvent(c->side, c->ev[1], 0));
    SCK((gemm<kStore>(c->side, H, H, B, c->d2, 1, H, c->a1, H, 1, gW2, H)));
    colsum_kernel<<<cdiv(H, 128), 128, 0, c->side>>>(c->d2, B, H, gb2);
    SCK(cudaGetLastError());
    SCK((gemm<kGeluGrad>(s, B, H, H, c->d2, H, 1, W2, H, 1, c->d1, H, nullptr, c->z1)));
    // layer 1
    SCK((gemm<kStore>(s, H, ni, B, c->d1, 1, H, x, ni, 1, gW1, ni)));
    colsum_kernel<<<cdiv(H, 128), 128, 0, s>>>(c->d1, B, H, gb1);
    SCK(cudaGetLastError());
    SCK(cudaEventRecord(c->ev[2], c->side));  // join
    SCK(cudaStreamWaitEvent(s, c->ev[2], 0));
    return SUR_OK;
}

// The Adam update; tick = false when the step counter was already advanced (training
// steps advance it in their gather kernel).
int adam(sur_ctx *c, cudaStream_t s, float lr, bool tick = true) {
    if (tick) tick_kernel<<<1, 1, 0, s>>>(c->tstep);
    adam_kernel<<<cdiv(c->np, 256), 256, 0, s>>>(c->p, c->g, c->m, c->v, c->np, c->tstep, lr, c->b1,
                                                c->b2, c->eps);
    SCK(cudaGetLastError());
    return SUR_OK;
}

}  // namespace

extern "C" {

const char *sur_last_error(const sur_ctx *c) { return c ? c->err.c_str() : ""; }

void sur_destroy(sur_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->epoch_graph) cudaGraphExecDestroy(c->epoch_graph);
    for (void *p : c->bufs) cudaFree(p);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    for (cudaEvent_t e : c->ev)
        if (e) cudaEventDestroy(e);
    delete c;
}

int sur_create(int32_t n_in, int32_t n_hidden, int32_t n_out, int32_t max_batch, uint64_t seed,
               void *stream, sur_ctx **out) {
    if (!out) return SUR_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_in < 1 || n_hidden < 1 || n_out < 1 || max_batch < 1 || n_in > 65536 || n_hidden > 65536 ||
        n_out > 65536)
        return SUR_ERR_INVALID_ARG;
    sur_ctx *c = new (std::nothrow) sur_ctx();
    if (!c) return SUR_ERR_ALLOC;
    c->nin = n_in;
    c->H = n_hidden;
    c->nout = n_out;
    c->max_batch = max_batch;
    c->stream = (cudaStream_t)stream;
    const long long sizes[6] = {(long long)n_hidden * n_in, n_hidden, (long long)n_hidden * n_hidden,
                                n_hidden, (long long)n_out * n_hidden, n_out};
    long long o = 0;
    for (int k = 0; k < 6; k++) {
        c->off[k] = o;
        o += (sizes[k] + 3) / 4 * 4;  // 16-byte aligned tensors
    }
    c->np = o;
    int rc = [&]() -> int {
        int r;
        const long long B = max_batch, H = n_hidden;
        if ((r = salloc(c, &c->p, c->np)) || (r = salloc(c, &c->g, c->np)) || (r = salloc(c, &c->m, c->np)) ||
            (r = salloc(c, &c->v, c->np)) || (r = salloc(c, &c->z1, B * H)) || (r = salloc(c, &c->a1, B * H)) ||
            (r = salloc(c, &c->z2, B * H)) || (r = salloc(c, &c->a2, B * H)) ||
            (r = salloc(c, &c->y, B * n_out)) || (r = salloc(c, &c->dy, B * n_out)) ||
            (r = salloc(c, &c->d2, B * H)) || (r = salloc(c, &c->d1, B * H)) ||
            (r = salloc(c, &c->xb, B * n_in)) || (r = salloc(c, &c->tb, B * n_out)) ||
            (r = salloc(c, &c->loss, 1)) || (r = salloc(c, &c->tstep, 1)))
            return r;
        // Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) initialisation from a seeded generator.
        std::vector<float> h(c->np, 0.0f);
        std::mt19937_64 gen(seed);
        const int fan[6] = {n_in, n_in, n_hidden, n_hidden, n_hidden, n_hidden};
        for (int k = 0; k < 6; k++) {
            std::uniform_real_distribution<float> U(-1.0f / std::sqrt((float)fan[k]), 1.0f / std::sqrt((float)fan[k]));
            for (long long i = 0; i < sizes[k]; i++) h[c->off[k] + i] = U(gen);
        }
        SCK(cudaMemcpy(c->p, h.data(), sizeof(float) * c->np, cudaMemcpyHostToDevice));
        SCK(cudaMemset(c->m, 0, sizeof(float) * c->np));
        SCK(cudaMemset(c->v, 0, sizeof(float) * c->np));
        SCK(cudaMemset(c->g, 0, sizeof(float) * c->np));
        SCK(cudaMemset(c->tstep, 0, sizeof(int)));
        SCK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
        SCK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
        for (cudaEvent_t &e : c->ev) SCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        SCK(gemm_setup());
        return SUR_OK;
    }();
    if (rc != SUR_OK) {
        sur_destroy(c);
        return rc;
    }
    *out = c;
    return SUR_OK;
}

int64_t sur_param_count(const sur_ctx *c) { return c ? (int64_t)c->np : -1; }

int sur_param_offsets(const sur_ctx *c, int64_t *offsets6) {
    if (!c || !offsets6) return SUR_ERR_INVALID_ARG;
    for (int k = 0; k < 6; k++) offsets6[k] = c->off[k];
    return SUR_OK;
}

int sur_set_params(sur_ctx *c, const float *host) {
    if (!c || !host) return SUR_ERR_INVALID_ARG;
    SCK(cudaMemcpyAsync(c->p, host, sizeof(float) * c->np, cudaMemcpyHostToDevice, c->stream));
    SCK(cudaMemsetAsync(c->m, 0, sizeof(float) * c->np, c->stream));
    SCK(cudaMemsetAsync(c->v, 0, sizeof(float) * c->np, c->stream));
    SCK(cudaMemsetAsync(c->tstep, 0, sizeof(int), c->stream));
    SCK(cudaStreamSynchronize(c->stream));
    return SUR_OK;
}

int sur_get_params(sur_ctx *c, float *host) {
    if (!c || !host) return SUR_ERR_INVALID_ARG;
    SCK(cudaMemcpyAsync(host, c->p, sizeof(float) * c->np, cudaMemcpyDeviceToHost, c->stream));
    SCK(cudaStreamSynchronize(c->stream));
    return SUR_OK;
}

int sur_forward(sur_ctx *c, const float *x_dev, int64_t B, float *y_dev) {
    if (!c || !x_dev || !y_dev || B < 0) return SUR_ERR_INVALID_ARG;
    for (int64_t b0 = 0; b0 < B; b0 += c->max_batch) {
        const int nb = (int)std::min<int64_t>(c->max_batch, B - b0);
        int rc = forward(c, c->stream, x_dev + b0 * c->nin, nb);
        if (rc != SUR_OK) return rc;
        SCK(cudaMemcpyAsync(y_dev + b0 * c->nout, c->y, sizeof(float) * nb * c->nout,
                            cudaMemcpyDeviceToDevice, c->stream));
    }
    return SUR_OK;
}

int sur_loss_grad(sur_ctx *c, const float *x_dev, const float *t_dev, int64_t B, float *loss_host,
                  float *grad_host) {
    if (!c || !x_dev || !t_dev || B < 1 || B > c->max_batch) return SUR_ERR_INVALID_ARG;
    int rc = backward(c, c->stream, x_dev, t_dev, (int)B, c->loss);
    if (rc != SUR_OK) return rc;
    if (loss_host) SCK(cudaMemcpyAsync(loss_host, c->loss, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    if (grad_host)
        SCK(cudaMemcpyAsync(grad_host, c->g, sizeof(float) * c->np, cudaMemcpyDeviceToHost, c->stream));
    SCK(cudaStreamSynchronize(c->stream));
    if (tc_faulted()) return sfail(c, SUR_ERR_CUDA, "a tensor-core product gave up waiting");
    return SUR_OK;
}

int sur_adam_step(sur_ctx *c, const float *x_dev, const float *t_dev, int64_t B, float lr) {
    if (!c || !x_dev || !t_dev || B < 1 || B > c->max_batch) return SUR_ERR_INVALID_ARG;
    int rc = backward(c, c->stream, x_dev, t_dev, (int)B, c->loss);
    if (rc != SUR_OK) return rc;
    return adam(c, c->stream, lr);
}

int sur_train(sur_ctx *c, const float *X_dev, const float *T_dev, int64_t n, int32_t batch,
              int32_t epochs, float lr, uint64_t seed, float *loss_host) {
    if (!c || !X_dev || !T_dev || n < 1 || batch < 1 || batch > c->max_batch || epochs < 0)
        return SUR_ERR_INVALID_ARG;
    const long long steps = n / batch;  // full mini-batches per epoch (the remainder is dropped)
    if (steps < 1) return sfail(c, SUR_ERR_INVALID_ARG, "fewer rows (%lld) than one mini-batch", (long long)n);
    if (c->perm_n < n) {
        int r = salloc(c, &c->perm, n);
        if (r) return r;
        c->perm_n = n;
    }
    if (c->loss_hist_n < steps) {
        int r = salloc(c, &c->loss_hist, steps);
        if (r) return r;
        c->loss_hist_n = steps;
    }
    const long long key[5] = {(long long)(size_t)X_dev, (long long)(size_t)T_dev, n, batch,
                              float_bits(lr)};
    bool same = c->epoch_graph != nullptr;
    for (int k = 0; k < 5; k++) same = same && key[k] == c->graph_key[k];
    if (!same) {
        if (c->epoch_graph) cudaGraphExecDestroy(c->epoch_graph);
        c->epoch_graph = nullptr;
        cudaGraph_t g = nullptr;
        SCK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
        int rc = SUR_OK;
        for (long long st = 0; st < steps && rc == SUR_OK; st++) {
            gather_step_kernel<<<cdiv((long long)batch * (c->nin + c->nout), 256), 256, 0, c->cap>>>(
                X_dev, T_dev, c->perm, (int)(st * batch), batch, c->nin, c->nout, c->xb, c->tb, c->tstep);
            rc = backward(c, c->cap, c->xb, c->tb, batch, c->loss_hist + st);
            if (rc == SUR_OK) rc = adam(c, c->cap, lr, false);
        }
        cudaError_t e = cudaStreamEndCapture(c->cap, &g);
        if (rc != SUR_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return sfail(c, SUR_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&c->epoch_graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return sfail(c, SUR_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
        for (int k = 0; k < 5; k++) c->graph_key[k] = key[k];
    }
    std::mt19937_64 gen(seed);
    std::vector<int> perm(n);
    std::vector<float> hist(steps);
    for (int ep = 0; ep < epochs; ep++) {
        for (long long i = 0; i < n; i++) perm[i] = (int)i;
        for (long long i = n - 1; i > 0; i--) {  // Fisher-Yates with the seeded generator
            std::uniform_int_distribution<long long> U(0, i);
            std::swap(perm[i], perm[U(gen)]);
        }
        SCK(cudaMemcpyAsync(c->perm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->stream));
        SCK(cudaGraphLaunch(c->epoch_graph, c->stream));
        if (loss_host) {
            SCK(cudaMemcpyAsync(hist.data(), c->loss_hist, sizeof(float) * steps, cudaMemcpyDeviceToHost,
                                c->stream));
            SCK(cudaStreamSynchronize(c->stream));
            if (tc_faulted()) return sfail(c, SUR_ERR_CUDA, "a tensor-core product gave up waiting");
            double s = 0.0;
            for (float x : hist) s += x;
            loss_host[ep] = (float)(s / steps);
        }
    }
    SCK(cudaStreamSynchronize(c->stream));
    if (tc_faulted()) return sfail(c, SUR_ERR_CUDA, "a tensor-core product gave up waiting");
    return SUR_OK;
}

int sur_loss(sur_ctx *c, const float *x_dev, const float *t_dev, int64_t B, float *loss_host) {
    if (!c || !x_dev || !t_dev || B < 1 || !loss_host) return SUR_ERR_INVALID_ARG;
    double acc = 0.0;
    for (int64_t b0 = 0; b0 < B; b0 += c->max_batch) {
        const int nb = (int)std::min<int64_t>(c->max_batch, B - b0);
        int rc = forward(c, c->stream, x_dev + b0 * c->nin, nb);
        if (rc != SUR_OK) return rc;
        mse_kernel<<<1, 256, 0, c->stream>>>(c->y, t_dev + b0 * c->nout, (long long)nb * c->nout, nullptr,
                                             c->loss);
        float l = 0.0f;
        SCK(cudaMemcpyAsync(&l, c->loss, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        SCK(cudaStreamSynchronize(c->stream));
        if (tc_faulted()) return sfail(c, SUR_ERR_CUDA, "a tensor-core product gave up waiting");
        acc += (double)l * nb;
    }
    *loss_host = (float)(acc / B);
    return SUR_OK;
}

int sur_fit_trust(sur_ctx *c, const float *X_dev, int64_t n, double q, double *radius_out) {
    if (!c || !X_dev || n < 1 || !(q > 0.0 && q <= 1.0)) return SUR_ERR_INVALID_ARG;
    double *norm_d = nullptr;
    if (cudaMalloc(&norm_d, sizeof(double) * (size_t)n) != cudaSuccess) {
        cudaGetLastError();
        return sfail(c, SUR_ERR_ALLOC, "%lld norms", (long long)n);
    }
    std::vector<double> norms((size_t)n);
    row_norm_kernel<<<(unsigned)cdiv(n * 32, 256), 256, 0, c->stream>>>(X_dev, n, c->nin, norm_d, -1.0, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(norms.data(), norm_d, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(norm_d);
    if (e != cudaSuccess) return sfail(c, SUR_ERR_CUDA, "training norms: %s", cudaGetErrorString(e));
    // the smallest norm with at least q n training norms at or below it
    const int64_t k = std::min<int64_t>(n, std::max<int64_t>(1, (int64_t)std::ceil(q * (double)n)));
    std::nth_element(norms.begin(), norms.begin() + (k - 1), norms.end());
    c->trust_radius = norms[(size_t)(k - 1)];
    if (radius_out) *radius_out = c->trust_radius;
    return SUR_OK;
}

int sur_trust(sur_ctx *c, const float *x_dev, int64_t B, int32_t *flags_dev) {
    if (!c || B < 0 || (B > 0 && (!x_dev || !flags_dev))) return SUR_ERR_INVALID_ARG;
    if (c->trust_radius < 0.0) return sfail(c, SUR_ERR_INVALID_ARG, "no trust radius (sur_fit_trust)");
    if (B == 0) return SUR_OK;
    row_norm_kernel<<<(unsigned)cdiv(B * 32, 256), 256, 0, c->stream>>>(x_dev, B, c->nin, nullptr,
                                                                        c->trust_radius, flags_dev);
    SCK(cudaGetLastError());
    return SUR_OK;
}

int sur_reconstruct(const float *coef_dev, const float *mean_dev, const float *phi_dev, int32_t B,
                    int64_t D, int32_t r, float *u_dev, void *stream) {
    if (!coef_dev || !mean_dev || !phi_dev || !u_dev || B < 0 || D < 0 || r < 1) return SUR_ERR_INVALID_ARG;
    reconstruct_kernel<<<cdiv((long long)B * D, 256), 256, 0, (cudaStream_t)stream>>>(coef_dev, mean_dev, phi_dev,
                                                                                      B, D, r, u_dev);
    return cudaGetLastError() == cudaSuccess ? SUR_OK : SUR_ERR_CUDA;
}

int sur_field_stats(const float *coef_dev, int32_t M, int32_t r, const float *mean_dev, const float *phi_dev,
                    int64_t D, float *work_dev, float *out_mean_dev, float *out_std_dev, void *stream) {
    if (!coef_dev || !mean_dev || !phi_dev || !work_dev || !out_mean_dev || !out_std_dev || M < 1 || r < 1 ||
        r > 64 || D < 0)
        return SUR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float *mu = work_dev, *C = work_dev + r;
    coef_mean_kernel<<<1, 64, 0, s>>>(coef_dev, M, r, mu);
    coef_cov_kernel<<<cdiv((long long)r * r, 256), 256, 0, s>>>(coef_dev, M, r, mu, C);
    field_stats_kernel<<<cdiv(D, 256), 256, sizeof(float) * (r + r * r), s>>>(mean_dev, phi_dev, D, r, mu, C,
                                                                              out_mean_dev, out_std_dev);
    return cudaGetLastError() == cudaSuccess ? SUR_OK : SUR_ERR_CUDA;
}

int sur_matmul(const float *A, int64_t sam, int64_t sak, const float *B, int64_t sbk, int64_t sbn,
               float *C, int32_t M, int32_t N, int32_t K, int32_t ldc, void *stream) {
    if (!A || !B || !C || M < 0 || N < 0 || K < 0 || ldc < N) return SUR_ERR_INVALID_ARG;
    if (gemm_setup() != cudaSuccess) return SUR_ERR_CUDA;
    return gemm<kStore>((cudaStream_t)stream, M, N, K, A, sam, sak, B, sbk, sbn, C, ldc) == cudaSuccess
               ? SUR_OK
               : SUR_ERR_CUDA;
}

}  // extern "C"
