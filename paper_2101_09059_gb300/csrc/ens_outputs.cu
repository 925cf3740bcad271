// Ensemble output statistics (Section 3: displacement-magnitude means and 5 %-95 % bands,
// displacement and stress time histories at chosen locations, stress components in the
// local cylindrical frame of the vessel).
//
// Quantities are formed on the device from the state of any precision form as binary64
// rows [rows][S] (sample index innermost):
//   displacement      rows (node, dof)                     [N][3][S]
//   |u|               rows node                           [N][S]
//   stress            rows (element, component)           [E][6][S]
// Stress (Section 2.2.1 and the transformation of Section 2.2.3): sigma_l = C(E) B u_l in
// the element frame, C with E_e,s the element mean of the nodal modulus (the average over
// the three Gauss points of the linear field), the plane-stress tensor rotated to the
// frame r = element normal, theta = r x t / |r x t|, z = t projected on the wall, with t
// the tangent of the centreline segment closest to the element centroid. Per element
// this is sigma_cyl = E_e,s W_e u_e (W_e: 6 x 9, built once in binary64), components
// (rr, theta theta, zz, r theta, rz, theta z).
//
// Statistics of a row: mean, sample variance (divisor S - 1) by the two-pass formula,
// and quantiles of type 7 (Hyndman and Fan): with the row sorted ascending, h = p (S - 1),
// j = floor h, Q(p) = x_j + (h - j)(x_{j+1} - x_j), evaluated without fused multiply-adds
// so that the result is the formula's. One warp owns a row and sorts it in shared memory
// (bitonic network).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "../../include/ens.h"
#include "ens_bits.cuh"
#include "ens_ctx.cuh"
#include "ens_internal.cuh"

namespace ens {
namespace {

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Value of state element (node i, dof d, sample s) as binary64, any form.
template <int FORM>
__device__ __forceinline__ double u_at(const void *u_main, const void *aux, int64_t idx) {
    if constexpr (FORM == kKahan32)
        return f32_to_f64(((const float *)u_main)[idx]) + f32_to_f64(((const float *)aux)[idx]);
    else if constexpr (FORM == kFP32Force)
        return join_state(((const float *)u_main)[idx], ((const uint32_t *)aux)[idx]);
    else
        return ((const double *)u_main)[idx];
}

// Running peak of |u| per node and sample (ens_set_peak), kept squared: after a step
// launch, the state just written has index n = *ctr + k_off + 1; when n is a multiple of
// the stride, peak2 = max(peak2, |u_n|^2). The binary32 forms form |u|^2 in binary32 from
// the words their forces gather (the FP32-force head, the compensated hi part: within one
// binary32 rounding of u), the FP64 form in binary64; the square root is taken when the
// peak is read (a binary64 square root per node and sample would occupy GB300's binary64
// pipe for longer than the step itself).
// A grid of a few blocks per SM strides over the node-samples, so that the launches after
// steps that record nothing retire at once.
template <int FORM>
__global__ void peak_kernel(const void *__restrict__ u_main, int32_t N, int32_t Sp,
                            const int64_t *__restrict__ ctr, int32_t k_off, int32_t stride,
                            double *__restrict__ peak2) {
    if ((*ctr + k_off + 1) % stride != 0) return;
    const uint32_t n = (uint32_t)N * (uint32_t)Sp;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const uint32_t i = t / (uint32_t)Sp;
        const size_t r0 = (size_t)i * 3 * Sp + (t - i * (uint32_t)Sp);
        double m2;
        if constexpr (FORM == kFP64) {
            const double *u = (const double *)u_main;
            const double x = u[r0], y = u[r0 + Sp], z = u[r0 + 2 * (size_t)Sp];
            m2 = x * x + y * y + z * z;
        } else {
            const float *u = (const float *)u_main;
            const float x = u[r0], y = u[r0 + Sp], z = u[r0 + 2 * (size_t)Sp];
            m2 = (double)(x * x + y * y + z * z);
        }
        if (m2 > peak2[t]) peak2[t] = m2;
    }
}

// rows [N][S] = sqrt(peak2) [N][Sp]
__global__ void peak_rows_kernel(const double *__restrict__ peak2, int32_t N, int32_t S, int32_t Sp,
                                 double *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * S) return;
    const int64_t i = t / S;
    out[t] = sqrt(peak2[i * Sp + (t - i * S)]);
}

// E_e,s = (E_a + E_b + E_c) / 3 over the element's nodes.
__global__ void ebar_kernel(const int32_t *__restrict__ tri, const double *__restrict__ En, int32_t E,
                            int32_t Sp, double *__restrict__ ebar) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)E * Sp) return;
    const int64_t e = t / Sp;
    const int32_t s = (int32_t)(t - e * Sp);
    const double a = En[(int64_t)tri[3 * e] * Sp + s], b = En[(int64_t)tri[3 * e + 1] * Sp + s],
                 c = En[(int64_t)tri[3 * e + 2] * Sp + s];
    ebar[t] = (a + b + c) / 3.0;
}

__device__ __forceinline__ void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ double dot3(const double *a, const double *b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// W_e = M_e C0 B_e Lambda_e (6 x 9, row-major) per element; counts elements whose
// centreline tangent is parallel to the wall normal into *bad.
__global__ void stress_operator_kernel(const double *__restrict__ xyz, const int32_t *__restrict__ tri,
                                       int32_t E, const double *__restrict__ pts, int32_t n_pts,
                                       double nu, double ks, double *__restrict__ W, int *bad) {
    const int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    double X[3][3];
    for (int a = 0; a < 3; a++)
        for (int k = 0; k < 3; k++) X[a][k] = xyz[3 * (int64_t)tri[3 * e + a] + k];
    double d12[3], d13[3], n[3], e1[3], e2[3];
    for (int k = 0; k < 3; k++) {
        d12[k] = X[1][k] - X[0][k];
        d13[k] = X[2][k] - X[0][k];
    }
    cross3(d12, d13, n);
    const double nn = sqrt(dot3(n, n)), l13 = sqrt(dot3(d13, d13));
    for (int k = 0; k < 3; k++) {
        n[k] /= nn;
        e1[k] = d13[k] / l13;  // in-plane axis along edge 1 -> 3 (any in-plane axis serves)
    }
    cross3(n, e1, e2);
    // local coordinates and the B matrix of Section 2.2.1 (rows exx, eyy, gxy, gxz, gyz)
    double x[3], y[3];
    for (int a = 0; a < 3; a++) {
        double r[3] = {X[a][0] - X[0][0], X[a][1] - X[0][1], X[a][2] - X[0][2]};
        x[a] = dot3(r, e1);
        y[a] = dot3(r, e2);
    }
    const double A2 = nn;  // twice the area
    const double by[3] = {(y[1] - y[2]) / A2, (y[2] - y[0]) / A2, (y[0] - y[1]) / A2};  // y23 y31 y12
    const double bx[3] = {(x[2] - x[1]) / A2, (x[0] - x[2]) / A2, (x[1] - x[0]) / A2};  // x32 x13 x21
    double B[5][9] = {};
    for (int a = 0; a < 3; a++) {
        B[0][3 * a] = by[a];
        B[1][3 * a + 1] = bx[a];
        B[2][3 * a] = bx[a];
        B[2][3 * a + 1] = by[a];
        B[3][3 * a + 2] = by[a];
        B[4][3 * a + 2] = bx[a];
    }
    // C / E
    const double f = 1.0 / (1.0 - nu * nu);
    const double C0[5] = {f, f, 0.5 * (1.0 - nu) * f, 0.5 * ks * (1.0 - nu) * f, 0.5 * ks * (1.0 - nu) * f};
    const double C01 = nu * f;  // (0,1) and (1,0)
    // cylindrical frame at the centroid
    double c[3];
    for (int k = 0; k < 3; k++) c[k] = (X[0][k] + X[1][k] + X[2][k]) / 3.0;
    double best = 1e300, t[3] = {0.0, 0.0, 1.0};
    for (int32_t p = 0; p + 1 < n_pts; p++) {
        const double *P0 = pts + 3 * p, *P1 = pts + 3 * (p + 1);
        double d[3] = {P1[0] - P0[0], P1[1] - P0[1], P1[2] - P0[2]};
        double w[3] = {c[0] - P0[0], c[1] - P0[1], c[2] - P0[2]};
        const double dd = dot3(d, d);
        if (!(dd > 0.0)) continue;
        double tau = dot3(w, d) / dd;
        tau = tau < 0.0 ? 0.0 : (tau > 1.0 ? 1.0 : tau);
        double q[3] = {w[0] - tau * d[0], w[1] - tau * d[1], w[2] - tau * d[2]};
        const double dist = dot3(q, q);
        if (dist < best) {
            best = dist;
            const double l = sqrt(dd);
            t[0] = d[0] / l;
            t[1] = d[1] / l;
            t[2] = d[2] / l;
        }
    }
    double th[3], zf[3];
    cross3(n, t, th);
    const double lt = sqrt(dot3(th, th));
    const double tr = dot3(t, n);
    for (int k = 0; k < 3; k++) zf[k] = t[k] - tr * n[k];
    const double lz = sqrt(dot3(zf, zf));
    double *We = W + (int64_t)e * 54;
    if (!(lt > 1e-8) || !(lz > 1e-8)) {
        atomicAdd(bad, 1);
        for (int k = 0; k < 54; k++) We[k] = 0.0;
        return;
    }
    for (int k = 0; k < 3; k++) {
        th[k] /= lt;
        zf[k] /= lz;
    }
    // frame vectors in local coordinates (e1, e2, n)
    const double *gv[3] = {n, th, zf};
    double lv[3][3];
    for (int a = 0; a < 3; a++) {
        lv[a][0] = dot3(gv[a], e1);
        lv[a][1] = dot3(gv[a], e2);
        lv[a][2] = dot3(gv[a], n);
    }
    // M (6 x 5): sigma_ab = a^T S_l b over the local components (xx, yy, xy, xz, yz)
    const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
    double M[6][5];
    for (int r = 0; r < 6; r++) {
        const double *a = lv[pa[r]], *b = lv[pb[r]];
        M[r][0] = a[0] * b[0];
        M[r][1] = a[1] * b[1];
        M[r][2] = a[0] * b[1] + a[1] * b[0];
        M[r][3] = a[0] * b[2] + a[2] * b[0];
        M[r][4] = a[1] * b[2] + a[2] * b[1];
    }
    // MC = M C0 (6 x 5), then MCB = MC B (6 x 9 in local dofs), then W = MCB Lambda_blk
    double MC[6][5];
    for (int r = 0; r < 6; r++) {
        MC[r][0] = M[r][0] * C0[0] + M[r][1] * C01;
        MC[r][1] = M[r][0] * C01 + M[r][1] * C0[1];
        MC[r][2] = M[r][2] * C0[2];
        MC[r][3] = M[r][3] * C0[3];
        MC[r][4] = M[r][4] * C0[4];
    }
    const double *lam[3] = {e1, e2, n};  // rows of Lambda: u_local = Lambda u_global
    for (int r = 0; r < 6; r++)
        for (int a = 0; a < 3; a++) {
            double row_l[3];  // coefficients of node a's local dofs
            for (int k = 0; k < 3; k++) {
                double sacc = 0.0;
                for (int q = 0; q < 5; q++) sacc += MC[r][q] * B[q][3 * a + k];
                row_l[k] = sacc;
            }
            for (int g = 0; g < 3; g++)
                We[r * 9 + 3 * a + g] = row_l[0] * lam[0][g] + row_l[1] * lam[1][g] + row_l[2] * lam[2][g];
        }
}

// Stress of element e, sample s into sig[6].
template <int FORM>
__device__ __forceinline__ void element_stress(const void *u_main, const void *aux, const int32_t *tri,
                                               const double *W, const double *ebar, int32_t Sp,
                                               int64_t e, int32_t s, double (&sig)[6]) {
    double u[9];
    for (int a = 0; a < 3; a++) {
        const int64_t node = tri[3 * e + a];
        for (int d = 0; d < 3; d++) u[3 * a + d] = u_at<FORM>(u_main, aux, (node * 3 + d) * Sp + s);
    }
    const double Es = ebar[e * Sp + s];
    const double *We = W + e * 54;
#pragma unroll
    for (int r = 0; r < 6; r++) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < 9; k++) acc = fma(__ldg(We + 9 * r + k), u[k], acc);
        sig[r] = Es * acc;
    }
}

template <int FORM>
__global__ void stress_rows_kernel(const void *u_main, const void *aux, const int32_t *__restrict__ tri,
                                   const double *__restrict__ W, const double *__restrict__ ebar,
                                   int32_t E, int32_t S, int32_t Sp, double *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)E * S) return;
    const int64_t e = t / S;
    const int32_t s = (int32_t)(t - e * S);
    double sig[6];
    element_stress<FORM>(u_main, aux, tri, W, ebar, Sp, e, s, sig);
    for (int r = 0; r < 6; r++) out[(e * 6 + r) * S + s] = sig[r];
}

template <int FORM>
__global__ void magnitude_rows_kernel(const void *u_main, const void *aux, int32_t N, int32_t S,
                                      int32_t Sp, double *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * S) return;
    const int64_t i = t / S;
    const int32_t s = (int32_t)(t - i * S);
    const double x = u_at<FORM>(u_main, aux, (i * 3 + 0) * Sp + s);
    const double y = u_at<FORM>(u_main, aux, (i * 3 + 1) * Sp + s);
    const double z = u_at<FORM>(u_main, aux, (i * 3 + 2) * Sp + s);
    out[t] = sqrt(x * x + y * y + z * z);
}

// One probe record: displacement of the probe nodes, stress of the probe elements.
template <int FORM>
__global__ void probe_record_kernel(const void *u_main, const void *aux, const int32_t *__restrict__ tri,
                                    const double *__restrict__ W, const double *__restrict__ ebar,
                                    int32_t S, int32_t Sp, const int32_t *__restrict__ pnodes, int32_t n_pn,
                                    const int32_t *__restrict__ pelems, int32_t n_pe,
                                    double *__restrict__ hu, double *__restrict__ hs) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n_u = (int64_t)n_pn * 3 * S;
    if (t < n_u) {
        const int64_t row = t / S;
        const int32_t s = (int32_t)(t - row * S);
        const int64_t node = pnodes[row / 3];
        hu[t] = u_at<FORM>(u_main, aux, (node * 3 + row % 3) * Sp + s);
        return;
    }
    const int64_t k = t - n_u;
    if (k >= (int64_t)n_pe * S) return;
    const int64_t p = k / S;
    const int32_t s = (int32_t)(k - p * S);
    double sig[6];
    element_stress<FORM>(u_main, aux, tri, W, ebar, Sp, pelems[p], s, sig);
    for (int r = 0; r < 6; r++) hs[(p * 6 + r) * S + s] = sig[r];
}

// Order-preserving map of binary64 bit patterns to unsigned 64-bit keys (negative values
// have every bit flipped, the others the sign bit), so the sort compares on the integer
// pipe; GB300 issues binary64 comparisons at the binary64 rate.
__device__ __forceinline__ uint64_t sort_key(double v) {
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    return b ^ ((b >> 63) ? ~0ull : 0x8000000000000000ull);
}
__device__ __forceinline__ double key_value(uint64_t k) {
    return __longlong_as_double((long long)(k ^ ((k >> 63) ? 0x8000000000000000ull : ~0ull)));
}

// Mean, sample variance and type-7 quantiles of every row; one warp per row, the row's
// sort keys in this warp's P words of shared memory (P = power of two >= S).
// inv_s = 1 / S, inv_s1 = 1 / (S - 1) (0 when S = 1) and s1 = S - 1 come from the host,
// which keeps divisions and conversions off GB300's binary64 pipe.
__global__ void row_stats_kernel(const double *__restrict__ rows, int64_t n_rows, int32_t S, int32_t P,
                                 double inv_s, double inv_s1, double s1, int32_t n_q,
                                 const double *__restrict__ q, double *__restrict__ mean,
                                 double *__restrict__ var, double *__restrict__ quant) {
    extern __shared__ uint64_t sm_keys[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint64_t *x = sm_keys + (size_t)wib * P;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; row < n_rows; row += warps) {
        const double *src = rows + row * S;
        double sum = 0.0;
        for (int32_t i = lane; i < P; i += 32) {
            const double v = i < S ? src[i] : INFINITY;
            x[i] = sort_key(v);
            if (i < S) sum += v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        const double mu = sum * inv_s;
        double ss = 0.0;
        for (int32_t i = lane; i < S; i += 32) {
            const double dlt = src[i] - mu;
            ss = fma(dlt, dlt, ss);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) {
            if (mean) mean[row] = mu;
            if (var) var[row] = ss * inv_s1;
        }
        if (quant && n_q > 0) {
            __syncwarp();
            for (int32_t k = 2; k <= P; k <<= 1)
                for (int32_t j = k >> 1; j > 0; j >>= 1) {
                    for (int32_t i = lane; i < P; i += 32) {
                        const int32_t ixj = i ^ j;
                        if (ixj > i) {
                            const uint64_t a = x[i], b = x[ixj];
                            if ((a > b) == ((i & k) == 0)) {
                                x[i] = b;
                                x[ixj] = a;
                            }
                        }
                    }
                    __syncwarp();
                }
            for (int32_t k = lane; k < n_q; k += 32) {
                const double h = __dmul_rn(q[k], s1);
                int32_t j = (int32_t)floor(h);
                if (j > S - 1) j = S - 1;
                if (j < 0) j = 0;
                const int32_t j1 = j + 1 < S ? j + 1 : S - 1;
                const double g = __dsub_rn(h, (double)j);
                const double xj = key_value(x[j]), xj1 = key_value(x[j1]);
                quant[row * n_q + k] = __dadd_rn(xj, __dmul_rn(g, __dsub_rn(xj1, xj)));
            }
        }
        __syncwarp();
    }
}

int pow2_at_least(int32_t S) {
    int P = 1;
    while (P < S) P <<= 1;
    return P;
}

}  // namespace

cudaError_t launch_element_mean(const int32_t *tri, const double *En, int32_t E, int32_t Sp, double *ebar,
                                cudaStream_t s) {
    const int64_t n = (int64_t)E * Sp;
    if (n == 0) return cudaSuccess;
    ebar_kernel<<<blocks_for(n, 256), 256, 0, s>>>(tri, En, E, Sp, ebar);
    return cudaGetLastError();
}

cudaError_t launch_peak(int form, const void *u_main, const void *aux, int32_t N, int32_t Sp,
                        const int64_t *step_ctr, int32_t k_off, int32_t stride, double *peak, cudaStream_t s) {
    (void)aux;
    const int64_t n = (int64_t)N * Sp;
    if (n == 0) return cudaSuccess;
    int dev = 0, sms = 0;  // multiprocessors of the current device
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1)
        sms = 148;
    const unsigned g = (unsigned)std::min<int64_t>(blocks_for(n, 256), (int64_t)sms * 8);
    if (form == kFP64)
        peak_kernel<kFP64><<<g, 256, 0, s>>>(u_main, N, Sp, step_ctr, k_off, stride, peak);
    else
        peak_kernel<kKahan32><<<g, 256, 0, s>>>(u_main, N, Sp, step_ctr, k_off, stride, peak);
    return cudaGetLastError();
}

// Rows statistics on the device (context free). Shared memory per warp: P doubles.
cudaError_t launch_row_stats(const double *rows, int64_t n_rows, int32_t S, int32_t n_q, const double *q_dev,
                             double *mean, double *var, double *quant, cudaStream_t s) {
    if (n_rows == 0) return cudaSuccess;
    const int P = pow2_at_least(S);
    int wpb = (int)std::max(1, std::min(8, (48 * 1024) / (P * 8)));
    size_t smem = (size_t)wpb * P * 8;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(row_stats_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = std::min<int64_t>((n_rows + wpb - 1) / wpb, 152 * 16);
    const double inv_s = 1.0 / (double)S, inv_s1 = S > 1 ? 1.0 / (double)(S - 1) : 0.0;
    row_stats_kernel<<<(unsigned)blocks, 32 * wpb, smem, s>>>(rows, n_rows, S, P, inv_s, inv_s1, (double)(S - 1),
                                                              n_q, q_dev, mean, var, quant);
    return cudaGetLastError();
}

}  // namespace ens

using namespace ens;

namespace {

int ofail(ens_ctx *c, int code, const char *msg) { return ctx_fail(c, code, "%s", msg); }

#define OCK(call)                                                                            \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) return ctx_fail(c, ENS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int64_t quantity_rows(const ens_ctx *c, int32_t qty) {
    if (qty == ENS_QTY_DISPLACEMENT) return (int64_t)c->N * 3;
    if (qty == ENS_QTY_DISP_MAGNITUDE) return c->N;
    if (qty == ENS_QTY_STRESS) return (int64_t)c->E * 6;
    if (qty == ENS_QTY_PEAK_MAGNITUDE) return c->N;
    return -1;
}

const void *aux_of(const ens_ctx *c) { return c->form == kFP32Force ? (const void *)c->utail : (const void *)c->ulo; }

template <int FORM>
cudaError_t launch_quantity_t(ens_ctx *c, int32_t qty, double *out) {
    const void *um = c->ug[c->cur], *ax = aux_of(c);
    if (qty == ENS_QTY_DISP_MAGNITUDE) {
        const int64_t n = (int64_t)c->N * c->S;
        magnitude_rows_kernel<FORM><<<blocks_for(n, 256), 256, 0, c->stream>>>(um, ax, c->N, c->S, c->Sp, out);
    } else {
        const int64_t n = (int64_t)c->E * c->S;
        stress_rows_kernel<FORM><<<blocks_for(n, 256), 256, 0, c->stream>>>(um, ax, c->tri_d, c->stress_w,
                                                                           c->ebar, c->E, c->S, c->Sp, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_quantity(ens_ctx *c, int32_t qty, double *out) {
    if (qty == ENS_QTY_DISPLACEMENT)
        return launch_export(c->form, c->ug[c->cur], aux_of(c), c->N, c->S, c->Sp, out, ENS_LAYOUT_NCS, c->stream);
    if (qty == ENS_QTY_PEAK_MAGNITUDE) {  // sqrt of the squared peak [N][Sp] -> rows [N][S]
        const int64_t n = (int64_t)c->N * c->S;
        if (n == 0) return cudaSuccess;
        peak_rows_kernel<<<blocks_for(n, 256), 256, 0, c->stream>>>(c->peak, c->N, c->S, c->Sp, out);
        return cudaGetLastError();
    }
    if (c->form == kFP64) return launch_quantity_t<kFP64>(c, qty, out);
    if (c->form == kFP32Force) return launch_quantity_t<kFP32Force>(c, qty, out);
    return launch_quantity_t<kKahan32>(c, qty, out);
}

template <int FORM>
cudaError_t launch_probe_t(ens_ctx *c, double *hu, double *hs) {
    const int64_t n = ((int64_t)c->probe_nn * 3 + c->probe_ne) * c->S;
    if (n == 0) return cudaSuccess;
    probe_record_kernel<FORM><<<blocks_for(n, 256), 256, 0, c->stream>>>(
        c->ug[c->cur], aux_of(c), c->tri_d, c->stress_w, c->ebar, c->S, c->Sp, c->probe_nodes, c->probe_nn,
        c->probe_elems, c->probe_ne, hu, hs);
    return cudaGetLastError();
}

}  // namespace

namespace ens {

// Record the current state at the probes if its step is a multiple of the stride and
// there is room (called by ens_step after every segment).
int probe_record(ens_ctx *c) {
    if (c->probe_stride <= 0 || c->step % c->probe_stride != 0 || c->probe_rec >= c->probe_cap) return ENS_OK;
    double *hu = c->probe_hu + (size_t)c->probe_rec * c->probe_nn * 3 * c->S;
    double *hs = c->probe_hs ? c->probe_hs + (size_t)c->probe_rec * c->probe_ne * 6 * c->S : nullptr;
    cudaError_t e = c->form == kFP64 ? launch_probe_t<kFP64>(c, hu, hs)
                    : c->form == kFP32Force ? launch_probe_t<kFP32Force>(c, hu, hs)
                                            : launch_probe_t<kKahan32>(c, hu, hs);
    if (e != cudaSuccess) return ctx_fail(c, ENS_ERR_CUDA, "probe record: %s", cudaGetErrorString(e));
    c->probe_steps.push_back(c->step);
    c->probe_rec++;
    return ENS_OK;
}

}  // namespace ens

extern "C" {

int ens_set_centerline(ens_ctx *c, int32_t n_pts, const double *pts) {
    if (!c) return ENS_ERR_INVALID_ARG;
    if (n_pts < 2 || !pts) return ofail(c, ENS_ERR_INVALID_ARG, "a centreline needs >= 2 points");
    for (int64_t k = 0; k < 3 * (int64_t)n_pts; k++)
        if (!std::isfinite(pts[k])) return ofail(c, ENS_ERR_INVALID_ARG, "centreline point not finite");
    double *pts_d = (double *)ctx_alloc(c, 8 * 3 * (size_t)n_pts);
    int *bad = (int *)ctx_alloc(c, sizeof(int));
    if (!c->stress_w) c->stress_w = (double *)ctx_alloc(c, 8 * 54 * (size_t)c->E);
    if (!pts_d || !bad || !c->stress_w) {
        if (pts_d) ctx_free(c, pts_d);
        if (bad) ctx_free(c, bad);
        return ofail(c, ENS_ERR_ALLOC, "centreline buffers");
    }
    int nbad = 0;
    cudaError_t e = cudaMemcpyAsync(pts_d, pts, 8 * 3 * (size_t)n_pts, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) {
        stress_operator_kernel<<<blocks_for(c->E, 128), 128, 0, c->stream>>>(c->xyz_d, c->tri_d, c->E, pts_d,
                                                                             n_pts, c->nu, c->ks, c->stress_w, bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    ctx_free(c, pts_d);
    ctx_free(c, bad);
    if (e != cudaSuccess) return ctx_fail(c, ENS_ERR_CUDA, "centreline: %s", cudaGetErrorString(e));
    if (nbad) {
        c->has_centerline = false;
        return ctx_fail(c, ENS_ERR_INVALID_ARG, "%d elements have a wall normal parallel to the centreline", nbad);
    }
    c->has_centerline = true;
    return ENS_OK;
}

int ens_quantity_device(ens_ctx *c, int32_t qty, double *out) {
    if (!c) return ENS_ERR_INVALID_ARG;
    const int64_t rows = quantity_rows(c, qty);
    if (rows < 0 || !out) return ofail(c, ENS_ERR_INVALID_ARG, "quantity code or output pointer");
    if (qty == ENS_QTY_STRESS && !c->has_centerline)
        return ofail(c, ENS_ERR_STATE, "stress needs a centreline (ens_set_centerline)");
    if (qty == ENS_QTY_PEAK_MAGNITUDE && !c->peak)
        return ofail(c, ENS_ERR_STATE, "no running peak (ens_set_peak)");
    OCK(launch_quantity(c, qty, out));
    return ENS_OK;
}

int ens_row_stats_device(int64_t n_rows, int32_t S, const double *rows, int32_t n_q, const double *q,
                         double *mean, double *var, double *quant, void *stream) {
    if (n_rows < 0 || S < 1 || S > 16384 || (n_rows > 0 && !rows) || n_q < 0 || n_q > 1024 ||
        (n_q > 0 && !q) || (n_q > 0 && !quant))
        return ENS_ERR_INVALID_ARG;
    for (int32_t k = 0; k < n_q; k++)
        if (!(q[k] >= 0.0 && q[k] <= 1.0)) return ENS_ERR_INVALID_ARG;
    if (n_rows == 0) return ENS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    double *q_d = nullptr;
    if (n_q > 0) {
        if (cudaMallocAsync((void **)&q_d, 8 * (size_t)n_q, s) != cudaSuccess) return ENS_ERR_ALLOC;
        if (cudaMemcpyAsync(q_d, q, 8 * (size_t)n_q, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            cudaFreeAsync(q_d, s);
            return ENS_ERR_CUDA;
        }
    }
    cudaError_t e = launch_row_stats(rows, n_rows, S, n_q, q_d, mean, var, n_q > 0 ? quant : nullptr, s);
    if (q_d) cudaFreeAsync(q_d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? ENS_OK : ENS_ERR_CUDA;
}

int ens_quantity_stats(ens_ctx *c, int32_t qty, int32_t n_q, const double *q, double *mean, double *var,
                       double *quant) {
    if (!c) return ENS_ERR_INVALID_ARG;
    const int64_t rows = quantity_rows(c, qty);
    if (rows < 0) return ofail(c, ENS_ERR_INVALID_ARG, "quantity code");
    if (n_q < 0 || n_q > 1024 || (n_q > 0 && (!q || !quant)))
        return ofail(c, ENS_ERR_INVALID_ARG, "quantile count or pointers");
    for (int32_t k = 0; k < n_q; k++)
        if (!(q[k] >= 0.0 && q[k] <= 1.0)) return ofail(c, ENS_ERR_INVALID_ARG, "quantile outside [0, 1]");
    if (c->S > 16384) return ofail(c, ENS_ERR_INVALID_ARG, "quantiles support S <= 16384");
    if (qty == ENS_QTY_STRESS && !c->has_centerline)
        return ofail(c, ENS_ERR_STATE, "stress needs a centreline (ens_set_centerline)");
    if (qty == ENS_QTY_PEAK_MAGNITUDE && !c->peak)
        return ofail(c, ENS_ERR_STATE, "no running peak (ens_set_peak)");
    const size_t need = (size_t)rows * c->S;
    if (c->qty_cap < need) {
        if (c->qty_buf) ctx_free(c, c->qty_buf);
        c->qty_buf = (double *)ctx_alloc(c, 8 * need);
        c->qty_cap = c->qty_buf ? need : 0;
        if (!c->qty_buf) return ofail(c, ENS_ERR_ALLOC, "quantity buffer");
    }
    const size_t sbytes = 8 * (size_t)rows * (2 + n_q) + 8 * (size_t)n_q;
    double *st = (double *)ctx_alloc(c, sbytes);
    if (!st) return ofail(c, ENS_ERR_ALLOC, "statistics buffer");
    double *m_d = st, *v_d = st + rows, *qt_d = st + 2 * rows, *q_d = qt_d + (size_t)rows * n_q;
    cudaError_t e = launch_quantity(c, qty, c->qty_buf);
    if (e == cudaSuccess && n_q > 0) e = cudaMemcpyAsync(q_d, q, 8 * (size_t)n_q, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_row_stats(c->qty_buf, rows, c->S, n_q, q_d, m_d, v_d, n_q > 0 ? qt_d : nullptr,
                                               c->stream);
    if (e == cudaSuccess && mean) e = cudaMemcpyAsync(mean, m_d, 8 * (size_t)rows, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && var) e = cudaMemcpyAsync(var, v_d, 8 * (size_t)rows, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && n_q > 0)
        e = cudaMemcpyAsync(quant, qt_d, 8 * (size_t)rows * n_q, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    ctx_free(c, st);
    if (e != cudaSuccess) return ctx_fail(c, ENS_ERR_CUDA, "quantity statistics: %s", cudaGetErrorString(e));
    return ENS_OK;
}

int ens_set_peak(ens_ctx *c, int32_t stride) {
    if (!c) return ENS_ERR_INVALID_ARG;
    if (stride < 0) return ofail(c, ENS_ERR_INVALID_ARG, "stride < 0");
    OCK(cudaStreamSynchronize(c->stream));
    if (c->peak) ctx_free(c, c->peak);
    c->peak = nullptr;
    c->peak_stride = 0;
    if (stride == 0) return ENS_OK;
    c->peak = (double *)ctx_alloc(c, 8 * (size_t)c->N * c->Sp);
    if (!c->peak) return ofail(c, ENS_ERR_ALLOC, "peak buffer");
    OCK(cudaMemsetAsync(c->peak, 0, 8 * (size_t)c->N * c->Sp, c->stream));
    OCK(cudaStreamSynchronize(c->stream));
    c->peak_stride = stride;
    return ENS_OK;
}

int ens_set_probes(ens_ctx *c, int32_t n_nodes, const int32_t *nodes, int32_t n_elems, const int32_t *elems,
                   int32_t stride, int64_t capacity) {
    if (!c) return ENS_ERR_INVALID_ARG;
    if (n_nodes < 0 || n_elems < 0 || (n_nodes > 0 && !nodes) || (n_elems > 0 && !elems) || stride < 0 ||
        capacity < 0 || (stride > 0 && capacity < 1) || (stride > 0 && n_nodes + n_elems == 0))
        return ofail(c, ENS_ERR_INVALID_ARG, "probe counts, pointers, stride or capacity");
    for (int32_t k = 0; k < n_nodes; k++)
        if (nodes[k] < 0 || nodes[k] >= c->N) return ofail(c, ENS_ERR_INVALID_ARG, "probe node id out of range");
    for (int32_t k = 0; k < n_elems; k++)
        if (elems[k] < 0 || elems[k] >= c->E) return ofail(c, ENS_ERR_INVALID_ARG, "probe element id out of range");
    if (n_elems > 0 && stride > 0 && !c->has_centerline)
        return ofail(c, ENS_ERR_STATE, "element probes need a centreline (ens_set_centerline)");
    void *old[] = {c->probe_nodes, c->probe_elems, c->probe_hu, c->probe_hs};
    for (void *p : old)
        if (p) ctx_free(c, p);
    c->probe_nodes = c->probe_elems = nullptr;
    c->probe_hu = c->probe_hs = nullptr;
    c->probe_stride = 0;
    c->probe_nn = c->probe_ne = 0;
    c->probe_rec = c->probe_cap = 0;
    c->probe_steps.clear();
    if (stride == 0) return ENS_OK;
    const size_t nu = (size_t)capacity * n_nodes * 3 * c->S, ns = (size_t)capacity * n_elems * 6 * c->S;
    c->probe_nodes = (int32_t *)ctx_alloc(c, 4 * (size_t)std::max(n_nodes, 1));
    c->probe_elems = (int32_t *)ctx_alloc(c, 4 * (size_t)std::max(n_elems, 1));
    c->probe_hu = (double *)ctx_alloc(c, 8 * std::max<size_t>(nu, 1));
    c->probe_hs = n_elems > 0 ? (double *)ctx_alloc(c, 8 * ns) : nullptr;
    if (!c->probe_nodes || !c->probe_elems || !c->probe_hu || (n_elems > 0 && !c->probe_hs))
        return ofail(c, ENS_ERR_ALLOC, "probe history buffers");
    if (n_nodes > 0) OCK(cudaMemcpyAsync(c->probe_nodes, nodes, 4 * (size_t)n_nodes, cudaMemcpyHostToDevice, c->stream));
    if (n_elems > 0) OCK(cudaMemcpyAsync(c->probe_elems, elems, 4 * (size_t)n_elems, cudaMemcpyHostToDevice, c->stream));
    OCK(cudaStreamSynchronize(c->stream));
    c->probe_nn = n_nodes;
    c->probe_ne = n_elems;
    c->probe_cap = capacity;
    c->probe_stride = stride;
    return ENS_OK;
}

int ens_get_probes(ens_ctx *c, double *u_out, double *sigma_out, int64_t *steps_out, int64_t *n_rec) {
    if (!c || !n_rec) return ENS_ERR_INVALID_ARG;
    *n_rec = c->probe_rec;
    if (c->probe_rec == 0) return ENS_OK;
    const size_t nu = (size_t)c->probe_rec * c->probe_nn * 3 * c->S;
    const size_t ns = (size_t)c->probe_rec * c->probe_ne * 6 * c->S;
    if (u_out && nu) OCK(cudaMemcpyAsync(u_out, c->probe_hu, 8 * nu, cudaMemcpyDeviceToHost, c->stream));
    if (sigma_out && ns) OCK(cudaMemcpyAsync(sigma_out, c->probe_hs, 8 * ns, cudaMemcpyDeviceToHost, c->stream));
    OCK(cudaStreamSynchronize(c->stream));
    if (steps_out)
        for (int64_t k = 0; k < c->probe_rec; k++) steps_out[k] = c->probe_steps[k];
    return ENS_OK;
}

}  // extern "C"
