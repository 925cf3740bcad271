// Proper orthogonal decomposition of solver snapshots on the device (sur_pod).
//
// The surrogate's outputs are POD coefficients of displacement fields the solver
// produced. With snapshots X [n][D] (binary32), mean m, centred X_c = X - m and the
// eigen-decomposition X_c X_c^T = V Lambda V^T (method of snapshots), the r leading modes
// are phi = X_c^T V_r Lambda_r^(-1/2) (orthonormal, D x r), the coefficients
// V_r Lambda_r^(1/2) = X_c phi, and the captured fraction sum_{k<r} lambda_k / trace.
//
// Device work: the column means (binary64 sums), the Gram matrix G = X_c X_c^T (binary32
// products of the centred values summed 32 at a time, the partial sums accumulated in
// binary64), subspace iteration on G in binary64 (block of b = r + 16 vectors: W = G Q,
// Cholesky-QR twice, Rayleigh-Ritz), and the mode projection phi = X_c^T V / sigma
// (binary64). The b x b problems (Gram of the block, its Cholesky factor, the symmetric
// eigenproblem of the Rayleigh quotient, by cyclic Jacobi rotations) are solved in this
// file's host code between the device steps.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sur.h"

namespace {

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// m[d] = (1/n) sum_i X[i][d] in binary64; mean32 = m rounded to binary32.
__global__ void pod_mean_kernel(const float *__restrict__ X, long long n, long long D, double *__restrict__ m,
                                float *__restrict__ mean32) {
    const long long d = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= D) return;
    double s = 0.0;
    for (long long i = 0; i < n; i++) s += (double)X[i * D + d];
    s /= (double)n;
    m[d] = s;
    mean32[d] = (float)s;
}

// G[i][j] = sum_d (X[i][d] - m[d]) (X[j][d] - m[d]) for one 64 x 64 tile (block (bi, bj),
// bi <= bj; the mirror tile is written too). The centred values are formed in binary64
// and rounded to binary32 in shared memory; each thread accumulates a 4 x 4 patch over 32
// values in binary32, then adds it to binary64 accumulators.
constexpr int kGT = 64, kGK = 32;
__global__ void __launch_bounds__(256) pod_gram_kernel(const float *__restrict__ X, const double *__restrict__ m,
                                                       long long n, long long D, double *__restrict__ G) {
    const int bi = blockIdx.y, bj = blockIdx.x;
    if (bi > bj) return;
    __shared__ float As[kGK][kGT + 4], Bs[kGK][kGT + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) acc[a][b] = 0.0;
    const long long i0 = (long long)bi * kGT, j0 = (long long)bj * kGT;
    for (long long d0 = 0; d0 < D; d0 += kGK) {
        // 64 rows x 32 columns of each operand: 2048 values, 8 per thread
        for (int t = threadIdx.x; t < kGT * kGK; t += 256) {
            const int r = t / kGK, k = t - r * kGK;
            const long long d = d0 + k;
            float a = 0.0f, b = 0.0f;
            if (d < D) {
                if (i0 + r < n) a = (float)((double)X[(i0 + r) * D + d] - m[d]);
                if (j0 + r < n) b = (float)((double)X[(j0 + r) * D + d] - m[d]);
            }
            As[k][r] = a;
            Bs[k][r] = b;
        }
        __syncthreads();
        float p[4][4] = {};
#pragma unroll 8
        for (int k = 0; k < kGK; k++) {
            float av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; a++) av[a] = As[k][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; b++) bv[b] = Bs[k][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = 0; b < 4; b++) p[a][b] = fmaf(av[a], bv[b], p[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 4; b++) acc[a][b] += (double)p[a][b];
        __syncthreads();
    }
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) {
            const long long i = i0 + ty * 4 + a, j = j0 + tx * 4 + b;
            if (i < n && j < n) {
                G[i * n + j] = acc[a][b];
                G[j * n + i] = acc[a][b];
            }
        }
}

// Z [n][b] = G [n][n] Q [n][b] in binary64 (thread per output; a warp shares the row of G).
__global__ void pod_gq_kernel(const double *__restrict__ G, const double *__restrict__ Q, long long n, int b,
                              double *__restrict__ Z) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * b) return;
    const long long i = t / b;
    const int c = (int)(t - i * b);
    const double *g = G + i * n;
    double s = 0.0;
    for (long long k = 0; k < n; k++) s = fma(g[k], Q[k * b + c], s);
    Z[t] = s;
}

// P [b][b] = A^T B for A, B [n][b] (one block per output pair, fixed reduction tree).
__global__ void pod_atb_kernel(const double *__restrict__ A, const double *__restrict__ B, long long n, int b,
                               double *__restrict__ P) {
    __shared__ double red[256];
    const int p = blockIdx.x / b, q = blockIdx.x - (blockIdx.x / b) * b;
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += 256) s = fma(A[i * b + p], B[i * b + q], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) P[blockIdx.x] = red[0];
}

// Y [n][b] = Z [n][b] M [b][b] (M row-major; used for Z R^-1 and for the Ritz rotations).
__global__ void pod_rmul_kernel(const double *__restrict__ Z, const double *__restrict__ M, long long n, int b,
                                double *__restrict__ Y) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * b) return;
    const long long i = t / b;
    const int c = (int)(t - i * b);
    double s = 0.0;
    for (int k = 0; k < b; k++) s = fma(Z[i * b + k], M[k * b + c], s);
    Y[t] = s;
}

// res[c] = sum_i (W[i][c] - theta[c] Q[i][c])^2 (one block per column).
__global__ void pod_residual_kernel(const double *__restrict__ W, const double *__restrict__ Q,
                                    const double *__restrict__ theta, long long n, int b, double *__restrict__ res) {
    __shared__ double red[256];
    const int c = blockIdx.x;
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += 256) {
        const double e = W[i * b + c] - theta[c] * Q[i * b + c];
        s = fma(e, e, s);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) res[c] = red[0];
}

// phi[d][k] = sum_i (X[i][d] - m[d]) V[i][k] / sigma[k] for k < r (V = the first r of the
// b columns of Q), binary64; thread per (d, group of 8 modes), V rows staged in shared
// memory 64 at a time.
__global__ void __launch_bounds__(128) pod_phi_kernel(const float *__restrict__ X, const double *__restrict__ m,
                                                      const double *__restrict__ Q, const double *__restrict__ sigma,
                                                      long long n, long long D, int b, int r,
                                                      float *__restrict__ phi) {
    __shared__ double Vs[64][8];
    const long long d = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int k0 = blockIdx.y * 8;
    double acc[8] = {};
    const double md = d < D ? m[d] : 0.0;
    for (long long i0 = 0; i0 < n; i0 += 64) {
        for (int t = threadIdx.x; t < 64 * 8; t += blockDim.x) {
            const int ii = t / 8, kk = t - (t / 8) * 8;
            Vs[ii][kk] = (i0 + ii < n && k0 + kk < r) ? Q[(i0 + ii) * b + k0 + kk] : 0.0;
        }
        __syncthreads();
        if (d < D) {
            const long long iend = n - i0 < 64 ? n - i0 : 64;
            for (long long ii = 0; ii < iend; ii++) {
                const double x = (double)X[(i0 + ii) * D + d] - md;
#pragma unroll
                for (int kk = 0; kk < 8; kk++) acc[kk] = fma(x, Vs[ii][kk], acc[kk]);
            }
        }
        __syncthreads();
    }
    if (d < D)
        for (int kk = 0; kk < 8; kk++)
            if (k0 + kk < r) phi[d * r + k0 + kk] = (float)(acc[kk] / sigma[k0 + kk]);
}

}  // namespace

namespace {

// Deterministic pseudo-random value in (-1, 1) of a 64-bit counter (SplitMix64 mixing).
double unit_hash(uint64_t k) {
    k += 0x9E3779B97F4A7C15ull;
    k = (k ^ (k >> 30)) * 0xBF58476D1CE4E5B9ull;
    k = (k ^ (k >> 27)) * 0x94D049BB133111EBull;
    k ^= k >> 31;
    return (double)(k >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// Upper Cholesky factor R of the symmetric b x b matrix B (B = R^T R), and its inverse M.
// Returns false when a pivot falls below 1e-12 of its diagonal entry (a block that is
// numerically rank-deficient).
bool cholesky_inverse(const std::vector<double> &B, int b, std::vector<double> &M) {
    std::vector<double> R((size_t)b * b, 0.0);
    for (int j = 0; j < b; j++) {
        double s = B[(size_t)j * b + j];
        for (int k = 0; k < j; k++) s -= R[(size_t)k * b + j] * R[(size_t)k * b + j];
        if (!(s > 1e-12 * B[(size_t)j * b + j]) || !(B[(size_t)j * b + j] > 0.0)) return false;
        const double d = std::sqrt(s);
        R[(size_t)j * b + j] = d;
        for (int i = j + 1; i < b; i++) {
            double t = B[(size_t)j * b + i];
            for (int k = 0; k < j; k++) t -= R[(size_t)k * b + j] * R[(size_t)k * b + i];
            R[(size_t)j * b + i] = t / d;
        }
    }
    M.assign((size_t)b * b, 0.0);
    for (int c = 0; c < b; c++)  // solve R x = e_c by back substitution
        for (int i = c; i >= 0; i--) {
            double t = (i == c) ? 1.0 : 0.0;
            for (int k = i + 1; k <= c; k++) t -= R[(size_t)i * b + k] * M[(size_t)k * b + c];
            M[(size_t)i * b + c] = t / R[(size_t)i * b + i];
        }
    return true;
}

// Orthonormal columns from Z [n][b] (row-major) by modified Gram-Schmidt, twice per column;
// a column left with less than 1e-10 of its length (linearly dependent) is replaced by a
// deterministic pseudo-random vector orthogonalised the same way.
void mgs2_refill(std::vector<double> &Z, int64_t n, int b, uint64_t salt) {
    for (int j = 0; j < b; j++) {
        for (int attempt = 0; attempt < 4; attempt++) {
            double n0 = 0.0;
            for (int64_t i = 0; i < n; i++) n0 += Z[(size_t)i * b + j] * Z[(size_t)i * b + j];
            for (int pass = 0; pass < 2; pass++)
                for (int k = 0; k < j; k++) {
                    double dot = 0.0;
                    for (int64_t i = 0; i < n; i++) dot += Z[(size_t)i * b + k] * Z[(size_t)i * b + j];
                    for (int64_t i = 0; i < n; i++) Z[(size_t)i * b + j] -= dot * Z[(size_t)i * b + k];
                }
            double nn = 0.0;
            for (int64_t i = 0; i < n; i++) nn += Z[(size_t)i * b + j] * Z[(size_t)i * b + j];
            if (nn > 1e-20 * n0 && nn > 0.0) {
                const double inv = 1.0 / std::sqrt(nn);
                for (int64_t i = 0; i < n; i++) Z[(size_t)i * b + j] *= inv;
                break;
            }
            for (int64_t i = 0; i < n; i++)
                Z[(size_t)i * b + j] = unit_hash(salt * 1000003ull + (uint64_t)attempt * 7919ull + (uint64_t)i * b + j);
        }
    }
}

// Eigenpairs of the symmetric b x b matrix A by cyclic Jacobi rotations: w descending,
// V [b][b] row-major with the eigenvectors as columns.
void jacobi_eigen(std::vector<double> A, int b, std::vector<double> &w, std::vector<double> &V) {
    V.assign((size_t)b * b, 0.0);
    for (int i = 0; i < b; i++) V[(size_t)i * b + i] = 1.0;
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0, tot = 0.0;
        for (int p = 0; p < b; p++)
            for (int q = 0; q < b; q++) {
                const double a = A[(size_t)p * b + q];
                tot += a * a;
                if (p != q) off += a * a;
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < b - 1; p++)
            for (int q = p + 1; q < b; q++) {
                const double apq = A[(size_t)p * b + q];
                if (apq == 0.0) continue;
                // rotation that annihilates A[p][q]: tan of the angle from the 2 x 2 block
                const double theta = (A[(size_t)q * b + q] - A[(size_t)p * b + p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < b; k++) {  // columns p, q
                    const double akp = A[(size_t)k * b + p], akq = A[(size_t)k * b + q];
                    A[(size_t)k * b + p] = c * akp - s * akq;
                    A[(size_t)k * b + q] = s * akp + c * akq;
                }
                for (int k = 0; k < b; k++) {  // rows p, q
                    const double apk = A[(size_t)p * b + k], aqk = A[(size_t)q * b + k];
                    A[(size_t)p * b + k] = c * apk - s * aqk;
                    A[(size_t)q * b + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < b; k++) {
                    const double vkp = V[(size_t)k * b + p], vkq = V[(size_t)k * b + q];
                    V[(size_t)k * b + p] = c * vkp - s * vkq;
                    V[(size_t)k * b + q] = s * vkp + c * vkq;
                }
            }
    }
    std::vector<int> order(b);
    for (int i = 0; i < b; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return A[(size_t)x * b + x] > A[(size_t)y * b + y]; });
    std::vector<double> V2((size_t)b * b);
    w.resize(b);
    for (int c = 0; c < b; c++) {
        w[c] = A[(size_t)order[c] * b + order[c]];
        for (int k = 0; k < b; k++) V2[(size_t)k * b + c] = V[(size_t)k * b + order[c]];
    }
    V.swap(V2);
}

struct PodBuffers {
    std::vector<void *> p;
    ~PodBuffers() {
        for (void *q : p) cudaFree(q);
    }
    template <typename T>
    bool get(T **out, size_t count) {
        void *q = nullptr;
        if (cudaMalloc(&q, sizeof(T) * std::max<size_t>(count, 1)) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        p.push_back(q);
        *out = (T *)q;
        return true;
    }
};

}  // namespace

extern "C" int sur_pod(const float *X_dev, int64_t n, int64_t D, int32_t r, float *mean_dev, float *phi_dev,
                       float *coef_dev, double *lam_host, double *frac_host, int32_t *iters_host, void *stream) {
    if (!X_dev || !mean_dev || !phi_dev || !coef_dev || n < 2 || n > 32768 || D < 1 || r < 1 || r > 48 ||
        r > n - 1)
        return SUR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int b = (int)std::min<int64_t>(n - 1, (int64_t)r + 16);  // X_c has rank n - 1 at most
    const size_t nb = (size_t)n * b;
    PodBuffers buf;
    double *m, *G, *Q, *Z, *W, *P, *M, *th, *res, *sig;
    if (!buf.get(&m, D) || !buf.get(&G, (size_t)n * n) || !buf.get(&Q, nb) || !buf.get(&Z, nb) ||
        !buf.get(&W, nb) || !buf.get(&P, (size_t)b * b) || !buf.get(&M, (size_t)b * b) || !buf.get(&th, b) ||
        !buf.get(&res, b) || !buf.get(&sig, r))
        return SUR_ERR_ALLOC;
#define PCK(call)                                                                                  \
    do {                                                                                           \
        if ((call) != cudaSuccess) return SUR_ERR_CUDA;                                            \
    } while (0)
    pod_mean_kernel<<<cdiv(D, 256), 256, 0, s>>>(X_dev, n, D, m, mean_dev);
    pod_gram_kernel<<<dim3(cdiv(n, kGT), cdiv(n, kGT)), 256, 0, s>>>(X_dev, m, n, D, G);
    PCK(cudaGetLastError());
    std::vector<double> diag((size_t)n), hq(nb), hP((size_t)b * b), hM, w, V, hres(b);
    PCK(cudaMemcpy2DAsync(diag.data(), sizeof(double), G, sizeof(double) * (size_t)(n + 1), sizeof(double),
                          (size_t)n, cudaMemcpyDeviceToHost, s));
    for (size_t k = 0; k < nb; k++) hq[k] = unit_hash(k);
    mgs2_refill(hq, n, b, 1);
    PCK(cudaMemcpyAsync(Q, hq.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, s));
    const unsigned gnb = cdiv((long long)nb, 256);
    auto gram_of = [&](const double *A, const double *B) -> int {  // hP = A^T B on the host
        pod_atb_kernel<<<b * b, 256, 0, s>>>(A, B, n, b, P);
        PCK(cudaGetLastError());
        PCK(cudaMemcpyAsync(hP.data(), P, sizeof(double) * b * b, cudaMemcpyDeviceToHost, s));
        PCK(cudaStreamSynchronize(s));
        return SUR_OK;
    };
    pod_gq_kernel<<<gnb, 256, 0, s>>>(G, Q, n, b, W);  // W = G Q
    const int max_it = 1000;
    int it = 0;
    int rc;
    for (it = 1; it <= max_it; it++) {
        // Rayleigh-Ritz on span(Q): H = Q^T G Q = V diag(w) V^T; Q <- Q V, W <- W V
        if ((rc = gram_of(Q, W)) != SUR_OK) return rc;
        for (int p = 0; p < b; p++)
            for (int q = p + 1; q < b; q++) {
                const double a = 0.5 * (hP[(size_t)p * b + q] + hP[(size_t)q * b + p]);
                hP[(size_t)p * b + q] = hP[(size_t)q * b + p] = a;
            }
        jacobi_eigen(hP, b, w, V);
        PCK(cudaMemcpyAsync(M, V.data(), sizeof(double) * b * b, cudaMemcpyHostToDevice, s));
        pod_rmul_kernel<<<gnb, 256, 0, s>>>(Q, M, n, b, Z);
        std::swap(Q, Z);
        pod_rmul_kernel<<<gnb, 256, 0, s>>>(W, M, n, b, Z);
        std::swap(W, Z);
        PCK(cudaMemcpyAsync(th, w.data(), sizeof(double) * b, cudaMemcpyHostToDevice, s));
        pod_residual_kernel<<<b, 256, 0, s>>>(W, Q, th, n, b, res);
        PCK(cudaGetLastError());
        PCK(cudaMemcpyAsync(hres.data(), res, sizeof(double) * b, cudaMemcpyDeviceToHost, s));
        PCK(cudaStreamSynchronize(s));
        const double scale = std::max(std::fabs(w[0]), 1e-300);
        bool conv = true;
        for (int c = 0; c < r; c++) conv = conv && std::sqrt(hres[c]) <= 1e-11 * scale;
        if (conv || it == max_it) break;
        // next block: orthonormalise W = G Q (Cholesky-QR twice; Gram-Schmidt on the host
        // when the block is numerically rank-deficient)
        bool ok = false;
        if ((rc = gram_of(W, W)) != SUR_OK) return rc;
        if (cholesky_inverse(hP, b, hM)) {
            PCK(cudaMemcpyAsync(M, hM.data(), sizeof(double) * b * b, cudaMemcpyHostToDevice, s));
            pod_rmul_kernel<<<gnb, 256, 0, s>>>(W, M, n, b, Q);
            if ((rc = gram_of(Q, Q)) != SUR_OK) return rc;
            if (cholesky_inverse(hP, b, hM)) {
                PCK(cudaMemcpyAsync(M, hM.data(), sizeof(double) * b * b, cudaMemcpyHostToDevice, s));
                pod_rmul_kernel<<<gnb, 256, 0, s>>>(Q, M, n, b, Z);
                std::swap(Q, Z);
                ok = true;
            }
        }
        if (!ok) {
            PCK(cudaMemcpyAsync(hq.data(), W, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
            PCK(cudaStreamSynchronize(s));
            mgs2_refill(hq, n, b, (uint64_t)it + 2);
            PCK(cudaMemcpyAsync(Q, hq.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, s));
        }
        pod_gq_kernel<<<gnb, 256, 0, s>>>(G, Q, n, b, W);
        PCK(cudaGetLastError());
    }
    // modes with the reference sign (largest-magnitude coefficient positive), coefficients
    // V_r sqrt(lambda), projections phi = X_c^T V_r / sqrt(lambda) (0 for a zero lambda)
    PCK(cudaMemcpyAsync(hq.data(), Q, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    PCK(cudaStreamSynchronize(s));
    std::vector<double> lam(r), sdiv(r);
    std::vector<float> coef((size_t)n * r);
    for (int c = 0; c < r; c++) {
        lam[c] = std::max(w[c], 0.0);
        int64_t j = 0;
        for (int64_t i = 1; i < n; i++)
            if (std::fabs(hq[(size_t)i * b + c]) > std::fabs(hq[(size_t)j * b + c])) j = i;
        if (hq[(size_t)j * b + c] < 0.0)
            for (int64_t i = 0; i < n; i++) hq[(size_t)i * b + c] = -hq[(size_t)i * b + c];
        const double sg = std::sqrt(lam[c]);
        sdiv[c] = sg > 0.0 ? sg : HUGE_VAL;
        for (int64_t i = 0; i < n; i++) coef[(size_t)i * r + c] = (float)(hq[(size_t)i * b + c] * sg);
    }
    PCK(cudaMemcpyAsync(Q, hq.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, s));
    PCK(cudaMemcpyAsync(sig, sdiv.data(), sizeof(double) * r, cudaMemcpyHostToDevice, s));
    PCK(cudaMemcpyAsync(coef_dev, coef.data(), sizeof(float) * coef.size(), cudaMemcpyHostToDevice, s));
    pod_phi_kernel<<<dim3(cdiv(D, 128), cdiv(r, 8)), 128, 0, s>>>(X_dev, m, Q, sig, n, D, b, r, phi_dev);
    PCK(cudaGetLastError());
    PCK(cudaStreamSynchronize(s));
#undef PCK
    double trace = 0.0, kept = 0.0;
    for (int64_t i = 0; i < n; i++) trace += diag[(size_t)i];
    for (int c = 0; c < r; c++) kept += lam[c];
    if (lam_host)
        for (int c = 0; c < r; c++) lam_host[c] = lam[c];
    if (frac_host) *frac_host = trace > 0.0 ? kept / trace : 1.0;
    if (iters_host) *iters_host = it;
    return SUR_OK;
}
