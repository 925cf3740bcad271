// The time-loop kernels: one fused launch per central-difference step, plus the
// ensemble statistics and the state export / import kernels.
//
// Step kernel (Section 2.3 Eq. dynamicsCD in velocity form, Section 2.4 assembly-free
// element products). One thread owns one node and V consecutive samples (a 16-byte
// vector along the ensemble), so the Q = Sp / V threads of a node read every state row
// as one coalesced segment. Per node the thread
//   1. gathers, through the node -> element list, the displacements of the other two
//      corners of every incident element and forms their offsets from its own node
//      (du = u_k - u_i);
//   2. applies the two 3 x 3 coupling blocks of the element matrix per unit E h to the
//      offsets and scales the result by the element's (E h)_e,s: since every row of the
//      element matrix annihilates rigid translations, K_e u_e for the node's rows equals
//      K_{c,a} du_a + K_{c,b} du_b, which needs 18 instead of 27 multiply-adds and removes
//      the cancellation of the (large) common translation;
//   3. sums the traction patterns with this step's amplitudes;
//   4. updates v and u with the lumped mass, the damping factor and the fixed-dof mask,
//      writing u_{n+1} to the other ping-pong buffer.
// There are no atomics in the force path: every node sums its own incidences in list
// order, so results are bitwise reproducible.
#include "ens_internal.cuh"

namespace ens {

namespace {

template <typename R> struct Vec16;
template <> struct Vec16<double> { using T = double2; };
template <> struct Vec16<float> { using T = float4; };

__device__ __forceinline__ void ld_nc(const double *p, double (&x)[2]) {
    double2 t = __ldg(reinterpret_cast<const double2 *>(p));
    x[0] = t.x;
    x[1] = t.y;
}
__device__ __forceinline__ void ld_nc(const float *p, float (&x)[4]) {
    float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    x[0] = t.x;
    x[1] = t.y;
    x[2] = t.z;
    x[3] = t.w;
}
__device__ __forceinline__ void ld_cs(const double *p, double (&x)[2]) {
    double2 t = __ldcs(reinterpret_cast<const double2 *>(p));
    x[0] = t.x;
    x[1] = t.y;
}
__device__ __forceinline__ void ld_cs(const float *p, float (&x)[4]) {
    float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
    x[0] = t.x;
    x[1] = t.y;
    x[2] = t.z;
    x[3] = t.w;
}
__device__ __forceinline__ void st_cs(double *p, const double (&x)[2]) {
    __stcs(reinterpret_cast<double2 *>(p), make_double2(x[0], x[1]));
}
__device__ __forceinline__ void st_cs(float *p, const float (&x)[4]) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(x[0], x[1], x[2], x[3]));
}
__device__ __forceinline__ void st_wb(double *p, const double (&x)[2]) {
    *reinterpret_cast<double2 *>(p) = make_double2(x[0], x[1]);
}
__device__ __forceinline__ void st_wb(float *p, const float (&x)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
}

// Coupling blocks of one incidence: 18 values.
__device__ __forceinline__ void ld_kc(const double *p, double (&k)[18]) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int r = 0; r < 9; r++) {
        double2 t = __ldg(q + r);
        k[2 * r] = t.x;
        k[2 * r + 1] = t.y;
    }
}
__device__ __forceinline__ void ld_kc(const float *p, float (&k)[18]) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int r = 0; r < 4; r++) {
        float4 t = __ldg(q + r);
        k[4 * r] = t.x;
        k[4 * r + 1] = t.y;
        k[4 * r + 2] = t.z;
        k[4 * r + 3] = t.w;
    }
    float2 t = __ldg(reinterpret_cast<const float2 *>(p + 16));
    k[16] = t.x;
    k[17] = t.y;
}

// Internal force of node i for samples [s0, s0 + V): f = sum over incidences of
// (E h)_e,s (K_{c,a} (u_a - u_i) + K_{c,b} (u_b - u_i)).
template <typename R>
__device__ __forceinline__ void node_force(const ForceView<R> &w, const R *__restrict__ ug,
                                           int32_t i, int32_t s0, const R (&ui)[3][Vw<R>::V],
                                           R (&f)[3][Vw<R>::V]) {
    constexpr int V = Vw<R>::V;
    const int64_t Sp = w.Sp;
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
        for (int v = 0; v < V; v++) f[d][v] = R(0);
    const int32_t p0 = __ldg(w.rowptr + i);
    const int32_t p1 = __ldg(w.rowptr + i + 1);
    for (int32_t p = p0; p < p1; ++p) {
        const int4 en = __ldg(w.ent + p);
        R ua[3][V], ub[3][V], e[V], k[18];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            ld_nc(ug + ((int64_t)en.y * 3 + d) * Sp + s0, ua[d]);
            ld_nc(ug + ((int64_t)en.z * 3 + d) * Sp + s0, ub[d]);
        }
        ld_nc(w.eh + (int64_t)en.x * Sp + s0, e);
        ld_kc(w.kc + (int64_t)p * Kc<R>::stride, k);
#pragma unroll
        for (int v = 0; v < V; v++) {
            const R a0 = ua[0][v] - ui[0][v], a1 = ua[1][v] - ui[1][v], a2 = ua[2][v] - ui[2][v];
            const R b0 = ub[0][v] - ui[0][v], b1 = ub[1][v] - ui[1][v], b2 = ub[2][v] - ui[2][v];
#pragma unroll
            for (int d = 0; d < 3; d++) {
                R t = k[3 * d] * a0;
                t = fma(k[3 * d + 1], a1, t);
                t = fma(k[3 * d + 2], a2, t);
                t = fma(k[9 + 3 * d], b0, t);
                t = fma(k[9 + 3 * d + 1], b1, t);
                t = fma(k[9 + 3 * d + 2], b2, t);
                f[d][v] = fma(e[v], t, f[d][v]);
            }
        }
    }
}

template <int FORM, typename R, bool FORCE_ONLY>
__global__ void __launch_bounds__(kBlock) step_kernel(const StepArgs<R> a) {
    constexpr int V = Vw<R>::V;
    const int32_t Q = a.fv.Q;
    const int64_t Sp = a.fv.Sp;
    const int64_t g = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    if (g >= (int64_t)a.fv.N * Q) return;
    const int32_t i = (int32_t)(g / Q);
    const int32_t s0 = (int32_t)(g - (int64_t)i * Q) * V;

    R ui[3][V];
#pragma unroll
    for (int d = 0; d < 3; d++) ld_nc(a.ug_cur + ((int64_t)i * 3 + d) * Sp + s0, ui[d]);
    R f[3][V];
    node_force<R>(a.fv, a.ug_cur, i, s0, ui, f);

    if constexpr (FORCE_ONLY) {
#pragma unroll
        for (int d = 0; d < 3; d++)
#pragma unroll
            for (int v = 0; v < V; v++)
                a.force_out[((int64_t)i * 3 + d) * Sp + s0 + v] = (double)f[d][v];
        return;
    } else {
        const int64_t n = *a.step_ctr + a.k_off;
        R fe[3] = {R(0), R(0), R(0)};
        for (int32_t j = 0; j < a.J; j++) {
            const R am = __ldg(a.amp + n * a.J + j);
            const R *P = a.modes + ((int64_t)j * a.fv.N + i) * 3;
#pragma unroll
            for (int d = 0; d < 3; d++) fe[d] = fma(am, __ldg(P + d), fe[d]);
        }
        R mi[V];
        ld_nc(a.minv + (int64_t)i * Sp + s0, mi);
        const unsigned fx = __ldg(a.fix + i);
        bool bad = false;
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const bool held = (fx >> d) & 1u;
            const int64_t row = ((int64_t)i * 3 + d) * Sp + s0;
            if constexpr (FORM == kFP64) {
                double vv[V], un[V];
                ld_cs(a.v64 + row, vv);
#pragma unroll
                for (int v = 0; v < V; v++) {
                    const double acc = (fe[d] - f[d][v]) * mi[v];
                    const double vn = held ? 0.0 : fma(a.c1, vv[v], a.c2 * acc);
                    un[v] = held ? 0.0 : fma(a.dt, vn, ui[d][v]);
                    vv[v] = vn;
                    bad |= !isfinite(un[v]);
                }
                st_cs(a.v64 + row, vv);
                st_wb(a.ug_next + row, un);
            } else if constexpr (FORM == kFP32Force) {
                double uu[4], vv[4];
                double h2[2];
                ld_cs(a.u64 + row, h2);
                uu[0] = h2[0];
                uu[1] = h2[1];
                ld_cs(a.u64 + row + 2, h2);
                uu[2] = h2[0];
                uu[3] = h2[1];
                ld_cs(a.v64 + row, h2);
                vv[0] = h2[0];
                vv[1] = h2[1];
                ld_cs(a.v64 + row + 2, h2);
                vv[2] = h2[0];
                vv[3] = h2[1];
                float ug[4];
                const float c2 = (float)a.c2;
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    const float acc = (fe[d] - f[d][v]) * mi[v];
                    const double vn = held ? 0.0 : fma(a.c1, vv[v], (double)(c2 * acc));
                    const double un = held ? 0.0 : fma(a.dt, vn, uu[v]);
                    vv[v] = vn;
                    uu[v] = un;
                    ug[v] = (float)un;
                    bad |= !isfinite(ug[v]);
                }
                st_cs(a.u64 + row, {uu[0], uu[1]});
                st_cs(a.u64 + row + 2, {uu[2], uu[3]});
                st_cs(a.v64 + row, {vv[0], vv[1]});
                st_cs(a.v64 + row + 2, {vv[2], vv[3]});
                st_wb(a.ug_next + row, ug);
            } else {  // kKahan32
                float lo[4], vv[4], hi[4];
                ld_cs(a.ulo + row, lo);
                ld_cs(a.v32 + row, vv);
                const float c1 = (float)a.c1, c2 = (float)a.c2, dt = (float)a.dt;
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    const float acc = (fe[d] - f[d][v]) * mi[v];
                    const float vn = held ? 0.0f : fmaf(c1, vv[v], c2 * acc);
                    // (hi, lo) += dt * vn as an error-free sum of hi and the small part.
                    const float y = fmaf(dt, vn, lo[v]);
                    const float s = ui[d][v] + y;
                    const float bb = s - ui[d][v];
                    const float err = (ui[d][v] - (s - bb)) + (y - bb);
                    hi[v] = held ? 0.0f : s;
                    lo[v] = held ? 0.0f : err;
                    vv[v] = vn;
                    bad |= !isfinite(s);
                }
                st_cs(a.ulo + row, lo);
                st_cs(a.v32 + row, vv);
                st_wb(a.ug_next + row, hi);
            }
        }
        if (bad) atomicOr(a.flags, 1);
    }
}

__global__ void advance_kernel(int64_t *ctr, int64_t n) { *ctr += n; }

// Value of sample s of state row `row` as binary64, for any form.
template <int FORM>
__device__ __forceinline__ double state_value(const void *u_main, const float *ulo, int64_t idx) {
    if constexpr (FORM == kKahan32)
        return (double)((const float *)u_main)[idx] + (double)ulo[idx];
    else
        return ((const double *)u_main)[idx];
}

// Ensemble mean and sample variance per dof: one warp per (node, dof) row, two passes
// (the second re-reads the row from cache), fixed reduction order.
template <int FORM>
__global__ void stats_kernel(const void *__restrict__ u_main, const float *__restrict__ ulo,
                             int32_t N, int32_t S, int32_t Sp, double *__restrict__ mean,
                             double *__restrict__ var) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= (int64_t)N * 3) return;
    const int64_t base = row * Sp;
    double s = 0.0;
    for (int32_t k = lane; k < S; k += 32) s += state_value<FORM>(u_main, ulo, base + k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double mu = s / (double)S;
    double q = 0.0;
    for (int32_t k = lane; k < S; k += 32) {
        const double x = state_value<FORM>(u_main, ulo, base + k) - mu;
        q = fma(x, x, q);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (lane == 0) {
        mean[row] = mu;
        var[row] = S > 1 ? q / (double)(S - 1) : 0.0;
    }
}

template <int FORM>
__global__ void export_kernel(const void *__restrict__ u_main, const float *__restrict__ ulo,
                              int32_t N, int32_t S, int32_t Sp, double *__restrict__ out,
                              int layout) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * 3 * S) return;
    const int64_t row = t / S;
    const int32_t s = (int32_t)(t - row * S);
    const double x = state_value<FORM>(u_main, ulo, row * Sp + s);
    if (layout == 0)
        out[(int64_t)s * N * 3 + row] = x;
    else
        out[t] = x;
}

// Load a binary64 [N][3][S] field into the gathered buffer (and the binary64 / low part
// state of the forms that keep one); padding samples are zero.
template <int FORM>
__global__ void import_kernel(const double *__restrict__ in, int32_t N, int32_t S, int32_t Sp,
                              void *ug, double *u64, float *ulo) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * 3 * Sp) return;
    const int64_t row = t / Sp;
    const int32_t s = (int32_t)(t - row * Sp);
    const double x = s < S ? in[row * S + s] : 0.0;
    if constexpr (FORM == kFP64) {
        ((double *)ug)[t] = x;
    } else if constexpr (FORM == kFP32Force) {
        ((float *)ug)[t] = (float)x;
        if (u64) u64[t] = x;
    } else {
        const float hi = (float)x;
        ((float *)ug)[t] = hi;
        if (ulo) ulo[t] = (float)(x - (double)hi);
    }
}

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

template <typename R>
cudaError_t launch_step(int form, const StepArgs<R> &a, bool force_only, cudaStream_t s) {
    const int64_t threads = (int64_t)a.fv.N * a.fv.Q;
    if (threads == 0) return cudaSuccess;
    const unsigned grid = blocks_for(threads, kBlock);
    if constexpr (sizeof(R) == 8) {
        if (force_only)
            step_kernel<kFP64, double, true><<<grid, kBlock, 0, s>>>(a);
        else
            step_kernel<kFP64, double, false><<<grid, kBlock, 0, s>>>(a);
    } else {
        if (force_only)
            step_kernel<kKahan32, float, true><<<grid, kBlock, 0, s>>>(a);
        else if (form == kFP32Force)
            step_kernel<kFP32Force, float, false><<<grid, kBlock, 0, s>>>(a);
        else
            step_kernel<kKahan32, float, false><<<grid, kBlock, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template cudaError_t launch_step<double>(int, const StepArgs<double> &, bool, cudaStream_t);
template cudaError_t launch_step<float>(int, const StepArgs<float> &, bool, cudaStream_t);

cudaError_t launch_advance(int64_t *step_ctr, int64_t n, cudaStream_t s) {
    advance_kernel<<<1, 1, 0, s>>>(step_ctr, n);
    return cudaGetLastError();
}

cudaError_t launch_stats(int form, const void *u_main, const float *ulo, int32_t N, int32_t S,
                         int32_t Sp, double *mean, double *var, cudaStream_t s) {
    const int64_t threads = (int64_t)N * 3 * 32;
    if (threads == 0) return cudaSuccess;
    const unsigned grid = blocks_for(threads, 256);
    if (form == kKahan32)
        stats_kernel<kKahan32><<<grid, 256, 0, s>>>(u_main, ulo, N, S, Sp, mean, var);
    else
        stats_kernel<kFP64><<<grid, 256, 0, s>>>(u_main, ulo, N, S, Sp, mean, var);
    return cudaGetLastError();
}

cudaError_t launch_export(int form, const void *u_main, const float *ulo, int32_t N, int32_t S,
                          int32_t Sp, double *out, int layout, cudaStream_t s) {
    const int64_t n = (int64_t)N * 3 * S;
    if (n == 0) return cudaSuccess;
    if (form == kKahan32)
        export_kernel<kKahan32><<<blocks_for(n, 256), 256, 0, s>>>(u_main, ulo, N, S, Sp, out,
                                                                   layout);
    else
        export_kernel<kFP64><<<blocks_for(n, 256), 256, 0, s>>>(u_main, ulo, N, S, Sp, out,
                                                                layout);
    return cudaGetLastError();
}

cudaError_t launch_import(int form, const double *in_ncs, int32_t N, int32_t S, int32_t Sp,
                          void *ug, double *u64, float *ulo, cudaStream_t s) {
    const int64_t n = (int64_t)N * 3 * Sp;
    if (n == 0) return cudaSuccess;
    const unsigned grid = blocks_for(n, 256);
    if (form == kFP64)
        import_kernel<kFP64><<<grid, 256, 0, s>>>(in_ncs, N, S, Sp, ug, u64, ulo);
    else if (form == kFP32Force)
        import_kernel<kFP32Force><<<grid, 256, 0, s>>>(in_ncs, N, S, Sp, ug, u64, ulo);
    else
        import_kernel<kKahan32><<<grid, 256, 0, s>>>(in_ncs, N, S, Sp, ug, u64, ulo);
    return cudaGetLastError();
}

}  // namespace ens
