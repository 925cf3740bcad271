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
#include <cstdio>
#include <utility>

#include "ens_bits.cuh"
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
__device__ __forceinline__ void ld_nc(const float *p, float (&x)[2]) {
    float2 t = __ldg(reinterpret_cast<const float2 *>(p));
    x[0] = t.x;
    x[1] = t.y;
}
__device__ __forceinline__ void ld_nc(const float *p, float (&x)[1]) { x[0] = __ldg(p); }
__device__ __forceinline__ void ld_nc(const double *p, double (&x)[1]) { x[0] = __ldg(p); }
__device__ __forceinline__ void ld_cs(const float *p, float (&x)[2]) {
    float2 t = __ldcs(reinterpret_cast<const float2 *>(p));
    x[0] = t.x;
    x[1] = t.y;
}
__device__ __forceinline__ void st_cs(float *p, const float (&x)[2]) {
    __stcs(reinterpret_cast<float2 *>(p), make_float2(x[0], x[1]));
}
__device__ __forceinline__ void st_wb(float *p, const float (&x)[2]) {
    *reinterpret_cast<float2 *>(p) = make_float2(x[0], x[1]);
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

__device__ __forceinline__ void ld_cs(const uint32_t *p, uint32_t (&x)[2]) {
    uint2 t = __ldcs(reinterpret_cast<const uint2 *>(p));
    x[0] = t.x;
    x[1] = t.y;
}
__device__ __forceinline__ void ld_cs(const uint32_t *p, uint32_t (&x)[4]) {
    uint4 t = __ldcs(reinterpret_cast<const uint4 *>(p));
    x[0] = t.x;
    x[1] = t.y;
    x[2] = t.z;
    x[3] = t.w;
}
__device__ __forceinline__ void st_cs(uint32_t *p, const uint32_t (&x)[2]) {
    __stcs(reinterpret_cast<uint2 *>(p), make_uint2(x[0], x[1]));
}
__device__ __forceinline__ void st_cs(uint32_t *p, const uint32_t (&x)[4]) {
    __stcs(reinterpret_cast<uint4 *>(p), make_uint4(x[0], x[1], x[2], x[3]));
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
// L2-only loads for data another SM may have written earlier in the same kernel (the
// persistent batched kernel); the read-only path is not coherent within a kernel.
__device__ __forceinline__ void ld_cg(const double *p, double (&x)[2]) {
    double2 t = __ldcg(reinterpret_cast<const double2 *>(p));
    x[0] = t.x;
    x[1] = t.y;
}
__device__ __forceinline__ void ld_cg(const float *p, float (&x)[4]) {
    float4 t = __ldcg(reinterpret_cast<const float4 *>(p));
    x[0] = t.x;
    x[1] = t.y;
    x[2] = t.z;
    x[3] = t.w;
}
__device__ __forceinline__ void ld_cg(const float *p, float (&x)[2]) {
    float2 t = __ldcg(reinterpret_cast<const float2 *>(p));
    x[0] = t.x;
    x[1] = t.y;
}
template <bool COH, typename R, int V>
__device__ __forceinline__ void ld_state(const R *p, R (&x)[V]) {
    if constexpr (COH)
        ld_cg(p, x);
    else
        ld_nc(p, x);
}

// The step index a block keeps in shared memory, read where it is used (a volatile load,
// so that it does not occupy registers through the force loop).
__device__ __forceinline__ int64_t lds_step(const void *p) {
    int64_t n;
    asm volatile("ld.shared.s64 %0, [%1];" : "=l"(n) : "r"(smem_addr(p)));
    return n;
}

// L2 prefetch of [p, p + bytes) widened to 16-byte boundaries (device allocations are
// padded to 256 bytes, so the widened range stays inside the array's allocation).
__device__ __forceinline__ void prefetch_range_l2(const void *p, uint32_t bytes) {
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p) & ~uintptr_t(15);
    const uintptr_t hi = (reinterpret_cast<uintptr_t>(p) + bytes + 15) & ~uintptr_t(15);
    bulk_prefetch_l2(reinterpret_cast<const void *>(lo), (uint32_t)(hi - lo));
}

// Per-thread bases of the gathered arrays: the thread's own column within node 0 of u and
// within (E h) row 0, so that a neighbour costs one 32 x 32 -> 64-bit multiply-add on its
// node (element) index, and its other two dof rows one row stride each.
template <typename R>
struct GatherBase {
    const char *u;   // ug + s0
    const char *eh;  // (E h) + s0
    int32_t node_b;  // 3 Sp sizeof(R)
    int32_t row_b;   // Sp sizeof(R)
    __device__ __forceinline__ GatherBase(const R *ug, const R *eh_, int32_t Sp, int32_t s0)
        : u(reinterpret_cast<const char *>(ug + s0)),
          eh(reinterpret_cast<const char *>(eh_ + s0)),
          node_b(3 * Sp * (int32_t)sizeof(R)),
          row_b(Sp * (int32_t)sizeof(R)) {}
    __device__ __forceinline__ const R *row(int32_t k, int d) const {
        return reinterpret_cast<const R *>(u + (int64_t)k * node_b + d * row_b);
    }
    __device__ __forceinline__ const R *ehrow(int32_t e) const {
        return reinterpret_cast<const R *>(eh + (int64_t)e * row_b);
    }
};

template <typename R, int V, bool COH = false>
__device__ __forceinline__ void node_force(const ForceView<R> &w, const R *__restrict__ ug,
                                           int32_t i, int32_t s0, const R (&ui)[3][V],
                                           R (&f)[3][V]) {
    const int64_t Sp = w.Sp;
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
        for (int v = 0; v < V; v++) f[d][v] = R(0);
    const GatherBase<R> g(ug, w.eh, (int32_t)Sp, s0);
    const int32_t p0 = __ldg(w.rowptr + i);
    const int32_t p1 = __ldg(w.rowptr + i + 1);
    for (int32_t p = p0; p < p1; ++p) {
        const int4 en = __ldg(w.ent + p);
        R ua[3][V], ub[3][V], e[V], k[18];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            ld_state<COH, R, V>(g.row(en.y, d), ua[d]);
            ld_state<COH, R, V>(g.row(en.z, d), ub[d]);
        }
        ld_nc(g.ehrow(en.x), e);
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

// Traction of node i at step n: sum_j amp[n][j] P_j[i] (sample-independent).
template <typename R>
__device__ __forceinline__ void node_traction(const StepArgs<R> &a, int32_t i, int64_t n,
                                              R (&fe)[3]) {
    fe[0] = fe[1] = fe[2] = R(0);
    for (int32_t j = 0; j < a.J; j++) {
        const R am = __ldg(a.amp + n * a.J + j);
        const R *P = a.modes + ((int64_t)j * a.fv.N + i) * 3;
#pragma unroll
        for (int d = 0; d < 3; d++) fe[d] = fma(am, __ldg(P + d), fe[d]);
    }
}

// Traction of node i at this launch's step (issued early so its loads overlap the gathers).
template <typename R>
__device__ __forceinline__ void step_traction(const StepArgs<R> &a, int32_t i, R (&fe)[3]) {
    node_traction<R>(a, i, *a.step_ctr + a.k_off, fe);
}

// The fused update of node i, samples [s0, s0 + V), one dof after the other (the shapes
// with two samples per thread, whose 48-register budget the loads of all three dofs at
// once would spill).
template <int FORM, typename R, int V>
__device__ __forceinline__ void node_update_per_dof(const StepArgs<R> &a, int32_t i, int32_t s0,
                                            const R (&ui)[3][V], const R (&f)[3][V],
                                            const R (&fe)[3]) {
    const int64_t Sp = a.fv.Sp;
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
            // binary64 u = (head ui, tail); the update runs in binary64, the bit splits and
            // the conversion of the binary32 velocity increment on the integer pipe. A held
            // dof is the same for every sample of the node, so the branch is uniform across
            // the node's threads.
            // The state rows are read whether or not the dof is held, so that these loads
            // do not wait for the fixed-dof mask.
            double vv[V], h2[2];
            uint32_t tl[V];
            float ug[V];
            ld_cs(a.utail + row, tl);
#pragma unroll
            for (int q = 0; q < V; q += 2) {
                ld_cs(a.v64 + row + q, h2);
                vv[q] = h2[0];
                vv[q + 1] = h2[1];
            }
            if (held) {
#pragma unroll
                for (int v = 0; v < V; v++) {
                    vv[v] = 0.0;
                    tl[v] = 0u;
                    ug[v] = 0.0f;
                }
            } else {
                const float c2 = a.c2f;
#pragma unroll
                for (int v = 0; v < V; v++) {
                    const float acc = (fe[d] - f[d][v]) * mi[v];
                    const double vn = fma(a.c1, vv[v], f32_to_f64_ftz(c2 * acc));
                    const double un = fma(a.dt, vn, join_state(ui[d][v], tl[v]));
                    vv[v] = vn;
                    bad |= !split_state(un, ug[v], tl[v]);
                }
            }
            st_cs(a.utail + row, tl);
#pragma unroll
            for (int q = 0; q < V; q += 2) st_cs(a.v64 + row + q, {vv[q], vv[q + 1]});
            st_wb(a.ug_next + row, ug);
        } else {  // kKahan32
            float lo[V], vv[V], hi[V];
            ld_cs(a.ulo + row, lo);  // read whether or not held, as above
            ld_cs(a.v32 + row, vv);
            if (held) {  // uniform across the node's threads
#pragma unroll
                for (int v = 0; v < V; v++) lo[v] = vv[v] = hi[v] = 0.0f;
            } else {
                const float c1 = a.c1f, c2 = a.c2f, dt = a.dtf;
#pragma unroll
                for (int v = 0; v < V; v++) {
                    const float acc = (fe[d] - f[d][v]) * mi[v];
                    const float vn = fmaf(c1, vv[v], c2 * acc);
                    // (hi, lo) += dt * vn as an error-free sum of hi and the small part.
                    const float y = fmaf(dt, vn, lo[v]);
                    const float s = ui[d][v] + y;
                    const float bb = s - ui[d][v];
                    hi[v] = s;
                    lo[v] = (ui[d][v] - (s - bb)) + (y - bb);
                    vv[v] = vn;
                    bad |= !isfinite(s);
                }
            }
            st_cs(a.ulo + row, lo);
            st_cs(a.v32 + row, vv);
            st_wb(a.ug_next + row, hi);
        }
    }
    if (bad) atomicOr(a.flags, 1);
}

// The fused update of node i, samples [s0, s0 + V): a = (f_ext - f_int) / m, then the
// velocity form of Eq. (dynamicsCD) with the fixed-dof mask, stored per form. Here every
// state word of the three dofs is loaded before the first store: the stores and the later
// dofs' loads go to different arrays, which the compiler cannot prove, so loading per dof
// serialises three round trips to memory.
template <int FORM, typename R, int V>
__device__ __forceinline__ void node_update_hoisted(const StepArgs<R> &a, int32_t i, int32_t s0,
                                            const R (&ui)[3][V], const R (&f)[3][V],
                                            const R (&fe)[3]) {
    const int64_t Sp = a.fv.Sp;
    R mi[V];
    ld_nc(a.minv + (int64_t)i * Sp + s0, mi);
    const unsigned fx = __ldg(a.fix + i);
    const int64_t row0 = (int64_t)i * 3 * Sp + s0;
    bool bad = false;
    if constexpr (FORM == kFP64) {
        double vv[3][V];
#pragma unroll
        for (int d = 0; d < 3; d++) ld_cs(a.v64 + row0 + d * Sp, vv[d]);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const bool held = (fx >> d) & 1u;
            const int64_t row = row0 + d * Sp;
            double un[V];
#pragma unroll
            for (int v = 0; v < V; v++) {
                const double acc = (fe[d] - f[d][v]) * mi[v];
                const double vn = held ? 0.0 : fma(a.c1, vv[d][v], a.c2 * acc);
                un[v] = held ? 0.0 : fma(a.dt, vn, ui[d][v]);
                vv[d][v] = vn;
                bad |= !isfinite(un[v]);
            }
            st_cs(a.v64 + row, vv[d]);
            st_wb(a.ug_next + row, un);
        }
    } else if constexpr (FORM == kFP32Force) {
        // binary64 u = (head ui, tail); the update runs in binary64, the bit splits and
        // the conversion of the binary32 velocity increment on the integer pipe. A held
        // dof is the same for every sample of the node, so the branch is uniform across
        // the node's threads; the state words are read whether or not the dof is held.
        double vv[3][V];
        uint32_t tl[3][V];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            ld_cs(a.utail + row0 + d * Sp, tl[d]);
#pragma unroll
            for (int q = 0; q < V; q += 2) {
                double h2[2];
                ld_cs(a.v64 + row0 + d * Sp + q, h2);
                vv[d][q] = h2[0];
                vv[d][q + 1] = h2[1];
            }
        }
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const bool held = (fx >> d) & 1u;
            const int64_t row = row0 + d * Sp;
            float ug[V];
            if (held) {
#pragma unroll
                for (int v = 0; v < V; v++) {
                    vv[d][v] = 0.0;
                    tl[d][v] = 0u;
                    ug[v] = 0.0f;
                }
            } else {
                const float c2 = a.c2f;
#pragma unroll
                for (int v = 0; v < V; v++) {
                    const float acc = (fe[d] - f[d][v]) * mi[v];
                    const double vn = fma(a.c1, vv[d][v], f32_to_f64_ftz(c2 * acc));
                    const double un = fma(a.dt, vn, join_state(ui[d][v], tl[d][v]));
                    vv[d][v] = vn;
                    bad |= !split_state(un, ug[v], tl[d][v]);
                }
            }
            st_cs(a.utail + row, tl[d]);
#pragma unroll
            for (int q = 0; q < V; q += 2) st_cs(a.v64 + row + q, {vv[d][q], vv[d][q + 1]});
            st_wb(a.ug_next + row, ug);
        }
    } else {  // kKahan32
        float lo[3][V], vv[3][V];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            ld_cs(a.ulo + row0 + d * Sp, lo[d]);  // read whether or not held, as above
            ld_cs(a.v32 + row0 + d * Sp, vv[d]);
        }
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const bool held = (fx >> d) & 1u;
            const int64_t row = row0 + d * Sp;
            float hi[V];
            if (held) {  // uniform across the node's threads
#pragma unroll
                for (int v = 0; v < V; v++) lo[d][v] = vv[d][v] = hi[v] = 0.0f;
            } else {
                const float c1 = a.c1f, c2 = a.c2f, dt = a.dtf;
#pragma unroll
                for (int v = 0; v < V; v++) {
                    const float acc = (fe[d] - f[d][v]) * mi[v];
                    const float vn = fmaf(c1, vv[d][v], c2 * acc);
                    // (hi, lo) += dt * vn as an error-free sum of hi and the small part.
                    const float y = fmaf(dt, vn, lo[d][v]);
                    const float sum = ui[d][v] + y;
                    const float bb = sum - ui[d][v];
                    hi[v] = sum;
                    lo[d][v] = (ui[d][v] - (sum - bb)) + (y - bb);
                    vv[d][v] = vn;
                    bad |= !isfinite(sum);
                }
            }
            st_cs(a.ulo + row, lo[d]);
            st_cs(a.v32 + row, vv[d]);
            st_wb(a.ug_next + row, hi);
        }
    }
    if (bad) atomicOr(a.flags, 1);
}

// The update used by every step kernel: the three dofs' loads issued together where the
// shape has the registers for them (four samples per thread), one dof after the other
// otherwise. Both evaluate the same operations (bitwise identical results).
template <int FORM, typename R, int V>
__device__ __forceinline__ void node_update(const StepArgs<R> &a, int32_t i, int32_t s0,
                                            const R (&ui)[3][V], const R (&f)[3][V],
                                            const R (&fe)[3]) {
    if constexpr (V >= 4)
        node_update_hoisted<FORM, R, V>(a, i, s0, ui, f, fe);
    else
        node_update_per_dof<FORM, R, V>(a, i, s0, ui, f, fe);
}

template <typename R, int V>
__device__ __forceinline__ void store_force(const StepArgs<R> &a, int32_t i, int32_t s0,
                                            const R (&f)[3][V]) {
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
        for (int v = 0; v < V; v++)
            a.force_out[((int64_t)i * 3 + d) * a.fv.Sp + s0 + v] = (double)f[d][v];
}

// Unstaged kernel: everything through the cache hierarchy (used when the staged plan
// does not apply).
template <int FORM, typename R, bool FORCE_ONLY, int V = Vw<R>::V>
__global__ void __launch_bounds__(kBlock) step_kernel(const StepArgs<R> a) {
    const int32_t Q = a.fv.Q;
    const int64_t Sp = a.fv.Sp;
    const int64_t g = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    if (g >= (int64_t)a.fv.N * Q) return;
    const int32_t i = (int32_t)(g / Q);
    const int32_t s0 = (int32_t)(g - (int64_t)i * Q) * V;
    R fe[3] = {R(0), R(0), R(0)};
    if constexpr (!FORCE_ONLY) step_traction<R>(a, i, fe);
    R ui[3][V];
#pragma unroll
    for (int d = 0; d < 3; d++) ld_nc(a.ug_cur + ((int64_t)i * 3 + d) * Sp + s0, ui[d]);
    R f[3][V];
    node_force<R, V>(a.fv, a.ug_cur, i, s0, ui, f);
    if constexpr (FORCE_ONLY)
        store_force<R, V>(a, i, s0, f);
    else
        node_update<FORM, R, V>(a, i, s0, ui, f, fe);
}

// Geometry update (Section 2.3, K(u) re-assembled on the deformed surface): the internal
// force with per-realisation corner blocks kcs [E][3][9][Sp] (block c = K_c,c+1 of the
// element), the same operations in the same order as node_force. Node i at corner c of
// element e couples to corner c + 1 through block c (read by rows) and to corner c + 2
// through K_c,c+2 = (K_c+2,c)^T, block c + 2 read by columns. Each block is read by the two
// corners it couples, neighbours in the node order, so the second read comes from L2.
template <typename R, int V>
__device__ __forceinline__ void node_force_geom(const ForceView<R> &w, const R *__restrict__ kcs,
                                                const R *__restrict__ ug, int32_t i, int32_t s0,
                                                const R (&ui)[3][V], R (&f)[3][V]) {
    const int64_t Sp = w.Sp;
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
        for (int v = 0; v < V; v++) f[d][v] = R(0);
    const GatherBase<R> g(ug, w.eh, (int32_t)Sp, s0);
    const int32_t p0 = __ldg(w.rowptr + i);
    const int32_t p1 = __ldg(w.rowptr + i + 1);
    for (int32_t p = p0; p < p1; ++p) {
        const int4 en = __ldg(w.ent + p);
        R da[3][V], db[3][V], e[V];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            ld_nc(g.row(en.y, d), da[d]);
            ld_nc(g.row(en.z, d), db[d]);
        }
        ld_nc(g.ehrow(en.x), e);
#pragma unroll
        for (int d = 0; d < 3; d++)
#pragma unroll
            for (int v = 0; v < V; v++) {
                da[d][v] -= ui[d][v];
                db[d][v] -= ui[d][v];
            }
        const int cz = en.w == 0 ? 2 : en.w - 1;
        const R *ky = kcs + ((int64_t)en.x * 3 + en.w) * 9 * Sp + s0;  // K_c,c+1, row d
        const R *kz = kcs + ((int64_t)en.x * 3 + cz) * 9 * Sp + s0;     // K_c+2,c, column d
#pragma unroll
        for (int d = 0; d < 3; d++) {
            R k0[V], k1[V], k2[V], k3[V], k4[V], k5[V];
            ld_nc(ky + (3 * d) * Sp, k0);
            ld_nc(ky + (3 * d + 1) * Sp, k1);
            ld_nc(ky + (3 * d + 2) * Sp, k2);
            ld_nc(kz + d * Sp, k3);
            ld_nc(kz + (3 + d) * Sp, k4);
            ld_nc(kz + (6 + d) * Sp, k5);
#pragma unroll
            for (int v = 0; v < V; v++) {
                R t = k0[v] * da[0][v];
                t = fma(k1[v], da[1][v], t);
                t = fma(k2[v], da[2][v], t);
                t = fma(k3[v], db[0][v], t);
                t = fma(k4[v], db[1][v], t);
                t = fma(k5[v], db[2][v], t);
                f[d][v] = fma(e[v], t, f[d][v]);
            }
        }
    }
}

template <int FORM, typename R, int V = Vw<R>::V>
__global__ void __launch_bounds__(kBlock) step_geom_kernel(const StepArgs<R> a) {
    const int32_t Q = a.fv.Q;
    const int64_t Sp = a.fv.Sp;
    const int64_t g = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    if (g >= (int64_t)a.fv.N * Q) return;
    const int32_t i = (int32_t)(g / Q);
    const int32_t s0 = (int32_t)(g - (int64_t)i * Q) * V;
    R fe[3] = {R(0), R(0), R(0)};
    step_traction<R>(a, i, fe);
    R ui[3][V];
#pragma unroll
    for (int d = 0; d < 3; d++) ld_nc(a.ug_cur + ((int64_t)i * 3 + d) * Sp + s0, ui[d]);
    R f[3][V];
    node_force_geom<R, V>(a.fv, a.kcs, a.ug_cur, i, s0, ui, f);
    // f_int(u_n) = K_m u_n + (f_int(u_m) - K_m u_m)
#pragma unroll
    for (int d = 0; d < 3; d++) {
        R cv[V];
        ld_nc(a.kcorr + ((int64_t)i * 3 + d) * Sp + s0, cv);
#pragma unroll
        for (int v = 0; v < V; v++) f[d][v] += cv[v];
    }
    node_update<FORM, R, V>(a, i, s0, ui, f, fe);
}

// (K_old - K_new) u at node i from the gathered words of u: K_old from the shared
// coupling blocks (scaled by (E h)) when kcs_old is null, else from the per-realisation
// corner blocks [E][3][9][Sp] read as in node_force_geom; K_new from kcs_new. Both
// stiffnesses scale by the same (E h), so the coefficient differences are taken first:
// the old and new coefficients are close, so their difference is exact or nearly so in
// the form's precision, and the result carries the rounding of the small difference
// force only, not the cancellation of two full forces.
template <typename R, int V>
__device__ __forceinline__ void node_force_delta(const ForceView<R> &w, const R *__restrict__ kcs_old,
                                                 const R *__restrict__ kcs_new, const R *__restrict__ ug, int32_t i,
                                                 int32_t s0, const R (&ui)[3][V], R (&f)[3][V]) {
    const int64_t Sp = w.Sp;
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
        for (int v = 0; v < V; v++) f[d][v] = R(0);
    const GatherBase<R> g(ug, w.eh, (int32_t)Sp, s0);
    const int32_t p0 = __ldg(w.rowptr + i);
    const int32_t p1 = __ldg(w.rowptr + i + 1);
    for (int32_t p = p0; p < p1; ++p) {
        const int4 en = __ldg(w.ent + p);
        R da[3][V], db[3][V], e[V];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            ld_nc(g.row(en.y, d), da[d]);
            ld_nc(g.row(en.z, d), db[d]);
        }
        ld_nc(g.ehrow(en.x), e);
#pragma unroll
        for (int d = 0; d < 3; d++)
#pragma unroll
            for (int v = 0; v < V; v++) {
                da[d][v] -= ui[d][v];
                db[d][v] -= ui[d][v];
            }
        const int cz = en.w == 0 ? 2 : en.w - 1;
        const int64_t oy = ((int64_t)en.x * 3 + en.w) * 9 * Sp + s0;  // K_c,c+1, row d
        const int64_t oz = ((int64_t)en.x * 3 + cz) * 9 * Sp + s0;     // K_c+2,c, column d
        const R *ks = w.kc + (int64_t)p * Kc<R>::stride;              // shared blocks of this incidence
#pragma unroll
        for (int d = 0; d < 3; d++) {
            // coefficient q of row d: q < 3 couples to corner y, q >= 3 to corner z
            const int64_t off[6] = {oy + (3 * d) * Sp, oy + (3 * d + 1) * Sp, oy + (3 * d + 2) * Sp,
                                    oz + d * Sp,       oz + (3 + d) * Sp,     oz + (6 + d) * Sp};
            R dk[6][V];
#pragma unroll
            for (int q = 0; q < 6; q++) {
                R kn[V];
                ld_nc(kcs_new + off[q], kn);
                if (kcs_old == nullptr) {
                    const R ko = __ldg(ks + (q < 3 ? 3 * d + q : 9 + 3 * d + (q - 3)));
#pragma unroll
                    for (int v = 0; v < V; v++) dk[q][v] = ko - kn[v];
                } else {
                    R ko[V];
                    ld_nc(kcs_old + off[q], ko);
#pragma unroll
                    for (int v = 0; v < V; v++) dk[q][v] = ko[v] - kn[v];
                }
            }
#pragma unroll
            for (int v = 0; v < V; v++) {
                R t = dk[0][v] * da[0][v];
                t = fma(dk[1][v], da[1][v], t);
                t = fma(dk[2][v], da[2][v], t);
                t = fma(dk[3][v], db[0][v], t);
                t = fma(dk[4][v], db[1][v], t);
                t = fma(dk[5][v], db[2][v], t);
                f[d][v] = fma(e[v], t, f[d][v]);
            }
        }
    }
}

// Geometry update, at a re-assembly on the state u = a.ug_cur: c64 += (K_old - K_new) u
// (shared blocks for K_old when kcs_old is null), from the words the step gathers. The
// increment is small next to the force, and its rounding with it, so the running sum in
// binary64 does not accumulate the binary32 forms' rounding of full forces; the step adds
// its rounding to binary32, cR.
template <typename R, int V>
__global__ void __launch_bounds__(kBlock) geo_correct_kernel(const StepArgs<R> a, const R *__restrict__ kcs_old,
                                                             const R *__restrict__ kcs_new, double *__restrict__ c64,
                                                             R *__restrict__ cR) {
    const int32_t Q = a.fv.Q;
    const int64_t Sp = a.fv.Sp;
    const int64_t g = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    if (g >= (int64_t)a.fv.N * Q) return;
    const int32_t i = (int32_t)(g / Q);
    const int32_t s0 = (int32_t)(g - (int64_t)i * Q) * V;
    R ui[3][V];
#pragma unroll
    for (int d = 0; d < 3; d++) ld_nc(a.ug_cur + ((int64_t)i * 3 + d) * Sp + s0, ui[d]);
    R df[3][V];
    node_force_delta<R, V>(a.fv, kcs_old, kcs_new, a.ug_cur, i, s0, ui, df);
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
        for (int v = 0; v < V; v++) {
            const int64_t idx = ((int64_t)i * 3 + d) * Sp + s0 + v;
            const double c = c64[idx] + (double)df[d][v];
            c64[idx] = c;
            cR[idx] = (R)c;
        }
}

// Staged kernel. Block b owns nodes [b nb, b nb + nb). One thread issues bulk copies
// (TMA, non-tensor) of the block's incidence entries, coupling blocks and own gathered
// displacement rows into shared memory, completing on one mbarrier, and asks L2 for the
// block's remaining state rows, which are only read after the force loop. Every thread
// then needs a single global round trip per incidence (the two other corners' rows and
// (E h)), with its own rows, the entry and the 18 coefficients coming from shared memory.
// One incidence of the force loop with everything it reads already in registers.
template <typename R, int V>
__device__ __forceinline__ void apply_incidence(const R (&ua)[3][V], const R (&ub)[3][V], const R (&e)[V],
                                                const R *__restrict__ k, const R (&ui)[3][V],
                                                R (&f)[3][V]) {
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

template <typename R, int V>
__device__ __forceinline__ void load_incidence(const GatherBase<R> &g, const int4 en,
                                               R (&ua)[3][V], R (&ub)[3][V], R (&e)[V]) {
#pragma unroll
    for (int d = 0; d < 3; d++) {
        ld_nc(g.row(en.y, d), ua[d]);
        ld_nc(g.row(en.z, d), ub[d]);
    }
    ld_nc(g.ehrow(en.x), e);
}

// REC: the block's entries and coupling blocks come from fixed-stride block records
// (StagePlan::rec_*), so thread 0 issues every bulk copy at once, without first loading
// the block's row offsets; each thread then reads its node's offsets from the staged
// record header.
template <int FORM, typename R, bool FORCE_ONLY, int BLOCK, int MINB, int V = Vw<R>::V,
          bool HOIST = false, bool REC = false>
__global__ void __launch_bounds__(BLOCK, MINB) step_staged_kernel(const StepArgs<R> a,
                                                                  const StagePlan pl) {
    const int32_t nb_block = pl.nb;
    const int32_t cnt_max = pl.cnt_max;
    const int32_t hw = REC ? pl.rec_h : 0;  // header words of a record
    constexpr int KS = Kc<R>::stride;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    int4 *rec_s = reinterpret_cast<int4 *>(smem + 16);
    int4 *ent_s = rec_s + hw;
    R *kc_s = reinterpret_cast<R *>(ent_s + cnt_max);
    R *ug_s = kc_s + (size_t)cnt_max * KS;

    grid_launch_dependents();  // the next step's blocks may stage their records early
    const int32_t Q = a.fv.Q;
    const int64_t Sp = a.fv.Sp;
    const int32_t N = a.fv.N;
    const int32_t n0 = blockIdx.x * nb_block;
    const int32_t nb = min(nb_block, N - n0);
    int32_t pb = 0, cnt = cnt_max;
    if constexpr (!REC) {
        pb = __ldg(a.fv.rowptr + n0);
        cnt = __ldg(a.fv.rowptr + n0 + nb) - pb;
        if (cnt < 1 || cnt > cnt_max) {
            // the plan does not describe this block: copy nothing, report, leave
            if (threadIdx.x == 0) atomicOr(a.flags, 4);
            return;
        }
    }
    const int32_t li = threadIdx.x / Q;
    const int32_t s0 = (threadIdx.x - li * Q) * V;
    const bool valid = li < nb;
    const int32_t i = n0 + li;
    int32_t p0 = 0, p1 = 0;
    if constexpr (!REC) {
        if (valid) {
            p0 = __ldg(a.fv.rowptr + i) - pb;
            p1 = __ldg(a.fv.rowptr + i + 1) - pb;
        }
    }
    const uint32_t row_bytes = (uint32_t)(nb * 3 * Sp * sizeof(R));
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
        const uint32_t b_ent = (uint32_t)(hw + cnt) * 16u;
        const uint32_t b_kc = (uint32_t)cnt * KS * (uint32_t)sizeof(R);
        mbar_expect_tx(bar, b_ent + b_kc + row_bytes);
        // the incidence records never change: staged before the previous step ends
        if constexpr (REC) {
            bulk_g2s(rec_s, pl.rec_ent + (size_t)blockIdx.x * (hw + cnt_max), b_ent, bar);
            bulk_g2s(kc_s, static_cast<const R *>(pl.rec_kc) + (size_t)blockIdx.x * cnt_max * KS, b_kc, bar);
        } else {
            bulk_g2s(ent_s, a.fv.ent + pb, b_ent, bar);
            bulk_g2s(kc_s, a.fv.kc + (size_t)pb * KS, b_kc, bar);
        }
    }
    grid_dependency_wait();  // the state below is written by the previous step
    if (threadIdx.x == 0) {
        bulk_g2s(ug_s, a.ug_cur + (size_t)n0 * 3 * Sp, row_bytes, bar);
        if constexpr (!FORCE_ONLY) {
            const size_t r0 = (size_t)n0 * 3 * Sp;
            bulk_prefetch_l2(a.minv + (size_t)n0 * Sp, (uint32_t)(nb * Sp * sizeof(R)));
            if constexpr (FORM == kKahan32) {
                bulk_prefetch_l2(a.ulo + r0, (uint32_t)(nb * 3 * Sp * 4));
                bulk_prefetch_l2(a.v32 + r0, (uint32_t)(nb * 3 * Sp * 4));
            } else if constexpr (FORM == kFP32Force) {
                bulk_prefetch_l2(a.utail + r0, (uint32_t)(nb * 3 * Sp * 4));
                bulk_prefetch_l2(a.v64 + r0, (uint32_t)(nb * 3 * Sp * 8));
            } else {
                bulk_prefetch_l2(a.v64 + r0, (uint32_t)(nb * 3 * Sp * 8));
            }
            // the block's traction-pattern rows (a few patterns only: one request each)
            if (a.J <= 4)
                for (int32_t j = 0; j < a.J; j++)
                    prefetch_range_l2(a.modes + ((int64_t)j * N + n0) * 3, (uint32_t)(nb * 3 * sizeof(R)));
            // the step index, once per block, while the copies are in flight (the
            // mbarrier uses the first 8 of the 16 bytes before the staged data)
            *reinterpret_cast<int64_t *>(smem + 8) = *a.step_ctr + a.k_off;
        }
    }
    __syncthreads();
    // HOIST: issue the traction loads now so they overlap the staging and the gathers
    R fe[3] = {R(0), R(0), R(0)};
    if constexpr (!FORCE_ONLY && HOIST)
        if (valid) node_traction<R>(a, i, lds_step(smem + 8), fe);
    if (!mbar_wait(bar, 0, kWaitLimit)) {
        // Report, then give the copies in flight one more bounded wait before leaving.
        if (threadIdx.x == 0) atomicOr(a.flags, 2);
        mbar_wait(bar, 0, kWaitLimit);
        return;
    }
    if (!valid) return;
    if constexpr (REC) {
        const int32_t *hdr = reinterpret_cast<const int32_t *>(rec_s);
        p0 = hdr[li];
        p1 = hdr[li + 1];
        if (p0 < 0 || p1 < p0 || p1 > cnt_max) {  // not a record of this plan
            atomicOr(a.flags, 4);
            return;
        }
    }

    R ui[3][V];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const R *src = ug_s + ((size_t)li * 3 + d) * Sp + s0;
#pragma unroll
        for (int v = 0; v < V; v++) ui[d][v] = src[v];
    }
    R f[3][V];
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
        for (int v = 0; v < V; v++) f[d][v] = R(0);
    const GatherBase<R> g(a.ug_cur, a.fv.eh, (int32_t)Sp, s0);
    for (int32_t p = p0; p < p1; ++p) {
        const int4 en = ent_s[p];
        R ua[3][V], ub[3][V], ev[V];
        load_incidence<R, V>(g, en, ua, ub, ev);
        apply_incidence<R, V>(ua, ub, ev, kc_s + (size_t)p * KS, ui, f);
    }
    if constexpr (FORCE_ONLY) {
        store_force<R, V>(a, i, s0, f);
    } else {
        if constexpr (!HOIST) node_traction<R>(a, i, lds_step(smem + 8), fe);
        node_update<FORM, R, V>(a, i, s0, ui, f, fe);
    }
}

// Persistent, double-buffered form of the staged kernel. Each CTA walks the node tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ...; thread 0 keeps the bulk copies (TMA) of the
// tile after next in flight in the other half of a two-buffer shared-memory ring while the
// block computes the current tile, so no block waits for its own staging after the first
// tile. Waits are bounded; all threads agree on the outcome through a block vote.
template <int FORM, typename R, int BLOCK, int MINB, int V>
__global__ void __launch_bounds__(BLOCK, MINB) step_pipelined_kernel(const StepArgs<R> a,
                                                                     const StagePlan pl,
                                                                     const int32_t n_tiles) {
    constexpr int KS = Kc<R>::stride;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    const int32_t Sp = a.fv.Sp, Q = a.fv.Q, N = a.fv.N;
    const int32_t nb_block = pl.nb, cnt_max = pl.cnt_max;
    const int32_t li = threadIdx.x / Q;
    const int32_t s0 = (threadIdx.x - li * Q) * V;
    auto stage_of = [&](int b) { return smem + 16 + (size_t)b * pl.stage; };
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
    }
    __syncthreads();
    // thread 0: stage tile `tile` into buffer `b` (entries, coupling blocks, own rows)
    auto issue = [&](int32_t tile, int b) -> bool {
        const int32_t n0 = tile * nb_block;
        const int32_t nb = min(nb_block, N - n0);
        const int32_t pb = __ldg(a.fv.rowptr + n0);
        const int32_t cnt = __ldg(a.fv.rowptr + n0 + nb) - pb;
        if (cnt < 1 || cnt > cnt_max) return false;
        // the block's generic-proxy reads of this buffer precede the bulk copies into it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        unsigned char *st = stage_of(b);
        int4 *ent_s = reinterpret_cast<int4 *>(st);
        R *kc_s = reinterpret_cast<R *>(ent_s + cnt_max);
        R *ug_s = kc_s + (size_t)cnt_max * KS;
        const uint32_t row_bytes = (uint32_t)(nb * 3 * Sp * sizeof(R));
        const uint32_t b_ent = (uint32_t)cnt * 16u;
        const uint32_t b_kc = (uint32_t)cnt * KS * (uint32_t)sizeof(R);
        mbar_expect_tx(&bars[b], b_ent + b_kc + row_bytes);
        bulk_g2s(ent_s, a.fv.ent + pb, b_ent, &bars[b]);
        bulk_g2s(kc_s, a.fv.kc + (size_t)pb * KS, b_kc, &bars[b]);
        bulk_g2s(ug_s, a.ug_cur + (size_t)n0 * 3 * Sp, row_bytes, &bars[b]);
        const size_t r0 = (size_t)n0 * 3 * Sp;
        const uint32_t rows = (uint32_t)nb * 3u * (uint32_t)Sp;
        bulk_prefetch_l2(a.minv + (size_t)n0 * Sp, (uint32_t)(nb * Sp * sizeof(R)));
        if constexpr (FORM == kKahan32) {
            bulk_prefetch_l2(a.ulo + r0, rows * 4u);
            bulk_prefetch_l2(a.v32 + r0, rows * 4u);
        } else if constexpr (FORM == kFP32Force) {
            bulk_prefetch_l2(a.utail + r0, rows * 4u);
            bulk_prefetch_l2(a.v64 + r0, rows * 8u);
        } else {
            bulk_prefetch_l2(a.v64 + r0, rows * 8u);
        }
        return true;
    };
    __shared__ int issued[2];
    if (threadIdx.x == 0) {
        issued[0] = blockIdx.x < n_tiles ? (issue(blockIdx.x, 0) ? 1 : -1) : 0;
        issued[1] = blockIdx.x + (int)gridDim.x < n_tiles ? (issue(blockIdx.x + gridDim.x, 1) ? 1 : -1) : 0;
    }
    __syncthreads();
    uint32_t uses[2] = {0u, 0u};
    int b = 0;
    for (int32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        bool ok = issued[b] == 1 && mbar_wait(&bars[b], uses[b] & 1u, kWaitLimit);
        ok = __syncthreads_and(ok);
        if (!ok) {
            // report, then give every copy in flight one more bounded wait before leaving
            if (threadIdx.x == 0) atomicOr(a.flags, issued[b] == -1 ? 4 : 2);
            for (int k = 0; k < 2; k++)
                if (issued[k] == 1) mbar_wait(&bars[k], uses[k] & 1u, kWaitLimit);
            return;
        }
        uses[b]++;
        const int32_t n0 = t * nb_block;
        const int32_t nb = min(nb_block, N - n0);
        const int32_t i = n0 + li;
        if (li < nb) {
            unsigned char *st = stage_of(b);
            const int4 *ent_s = reinterpret_cast<const int4 *>(st);
            const R *kc_s = reinterpret_cast<const R *>(ent_s + cnt_max);
            const R *ug_s = kc_s + (size_t)cnt_max * KS;
            const int32_t pb = __ldg(a.fv.rowptr + n0);
            const int32_t p0 = __ldg(a.fv.rowptr + i) - pb, p1 = __ldg(a.fv.rowptr + i + 1) - pb;
            R ui[3][V];
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const R *src = ug_s + ((size_t)li * 3 + d) * Sp + s0;
#pragma unroll
                for (int v = 0; v < V; v++) ui[d][v] = src[v];
            }
            R f[3][V];
#pragma unroll
            for (int d = 0; d < 3; d++)
#pragma unroll
                for (int v = 0; v < V; v++) f[d][v] = R(0);
            const GatherBase<R> g(a.ug_cur, a.fv.eh, Sp, s0);
            for (int32_t p = p0; p < p1; ++p) {
                const int4 en = ent_s[p];
                R ua[3][V], ub[3][V], ev[V];
                load_incidence<R, V>(g, en, ua, ub, ev);
                apply_incidence<R, V>(ua, ub, ev, kc_s + (size_t)p * KS, ui, f);
            }
            R fe[3];
            step_traction<R>(a, i, fe);
            node_update<FORM, R, V>(a, i, s0, ui, f, fe);
        }
        __syncthreads();  // the whole block is done with buffer b
        if (threadIdx.x == 0) {
            const int32_t next = t + 2 * (int32_t)gridDim.x;
            issued[b] = next < n_tiles ? (issue(next, b) ? 1 : -1) : 0;
        }
        __syncthreads();
        b ^= 1;
    }
}

__global__ void advance_kernel(int64_t *ctr, int64_t n) { *ctr += n; }

// Deterministic non-zero values of magnitude <= scale (an integer hash of the index).
__global__ void fill_kernel(void *p, int64_t n, int is_double, float scale, uint32_t seed) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    uint32_t h = (uint32_t)t * 2654435761u ^ seed;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    const float v = scale * ((float)(h >> 8) * (1.0f / 16777216.0f) - 0.5f);
    if (is_double)
        ((double *)p)[t] = (double)v;
    else
        ((float *)p)[t] = v;
}

__global__ void advance_many_kernel(int64_t *const *ctrs, int32_t n, int64_t by) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) *ctrs[k] += by;
}

// One tile of a batched launch: member item.x, nodes from item.y, lanes from item.z.
// The tile holds BLOCK / Qt nodes with Qt = min(Q, BLOCK) threads per node.
template <int FORM, typename R, int BLOCK, bool COH>
__device__ __forceinline__ void batch_tile(const MemberDev<R> *__restrict__ mem, const int4 item,
                                           int32_t k_off, int *flags) {
    constexpr int V = Vw<R>::V;
    const MemberDev<R> &m = mem[item.x];
    const int32_t Q = m.fv.Q;
    const int32_t Qt = Q < BLOCK ? Q : BLOCK;
    const int32_t li = threadIdx.x / Qt;
    const int32_t q = item.z + (threadIdx.x - li * Qt);
    const int32_t i = item.y + li;
    if (li >= BLOCK / Qt || i >= m.fv.N || q >= Q) return;
    StepArgs<R> a;
    a.fv = m.fv;
    const int par = m.cur ^ (k_off & 1);
    a.ug_cur = m.ug[par];
    a.ug_next = const_cast<R *>(m.ug[par ^ 1]);
    a.utail = m.utail;
    a.v64 = m.v64;
    a.ulo = m.ulo;
    a.v32 = m.v32;
    a.minv = m.minv;
    a.fix = m.fix;
    a.modes = m.modes;
    a.amp = m.amp;
    a.step_ctr = m.step_ctr;
    a.k_off = k_off;
    a.J = m.J;
    const bool start = m.first && k_off == 0;
    a.c1 = start ? m.c1s : m.c1;
    a.c2 = start ? m.c2s : m.c2;
    a.dt = m.dt;
    a.c1f = (float)a.c1;
    a.c2f = (float)a.c2;
    a.dtf = (float)a.dt;
    a.force_out = nullptr;
    a.flags = flags;
    const int32_t s0 = q * V;
    const int64_t Sp = m.fv.Sp;
    R ui[3][V];
#pragma unroll
    for (int d = 0; d < 3; d++) ld_state<COH, R, V>(a.ug_cur + ((int64_t)i * 3 + d) * Sp + s0, ui[d]);
    R fe[3];
    step_traction<R>(a, i, fe);
    R f[3][V];
    node_force<R, V, COH>(a.fv, a.ug_cur, i, s0, ui, f);
    node_update<FORM, R, V>(a, i, s0, ui, f, fe);
}

// Batched step: one launch advances every member one step (graph-captured in chunks).
template <int FORM, typename R, int BLOCK>
__global__ void __launch_bounds__(BLOCK) batch_step_kernel(const MemberDev<R> *__restrict__ mem,
                                                           const int4 *__restrict__ items,
                                                           int32_t k_off, int *flags) {
    batch_tile<FORM, R, BLOCK, false>(mem, items[blockIdx.x], k_off, flags);
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Persistent batched kernel: n_steps steps in one cooperative launch. Every block keeps
// the same tiles (round robin) for the whole launch; a grid barrier with a bounded spin
// separates the steps. Displacement rows written by other blocks are read through L2.
template <int FORM, typename R, int BLOCK>
__global__ void __launch_bounds__(BLOCK) batch_persistent_kernel(
    const MemberDev<R> *__restrict__ mem, const int4 *__restrict__ items, int32_t n_items,
    int32_t n_steps, unsigned *bar, int *flags) {
    __shared__ int abort_all;
    for (int32_t k = 0; k < n_steps; k++) {
        for (int32_t t = blockIdx.x; t < n_items; t += gridDim.x)
            batch_tile<FORM, R, BLOCK, true>(mem, items[t], k, flags);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(bar, 1u);
            const unsigned target = (unsigned)(k + 1) * gridDim.x;
            bool ok = false;
            for (uint32_t it = 0; it < kSpinLimit; ++it) {
                if (ld_acquire(bar) >= target) {
                    ok = true;
                    break;
                }
                __nanosleep(64);
            }
            if (!ok) atomicOr(flags, 2);
            abort_all = ok ? 0 : 1;
            __threadfence();
        }
        __syncthreads();
        if (abort_all) return;
    }
}

// Ensemble mean and sample variance per dof: 8 lanes per (node, dof) row, each lane
// holding up to 16 of the row's samples in registers between the two passes (exact
// two-pass formula; the shuffle tree fixes the reduction order). For wider ensembles
// the second pass re-reads the row from cache. The binary32 pair of the compensated
// form is widened on the integer pipe. inv_s = 1 / S, inv_s1 = 1 / (S - 1) (0 if S = 1).
constexpr int kStatLanes = 8;
constexpr int kStatRegs = 16;

// Value of sample s of state row `row` as binary64, for any form (aux: the compensated
// form's low parts, or the FP32-force form's tails), integer-pipe conversions.
template <int FORM>
__device__ __forceinline__ double state_value_fast(const void *u_main, const void *aux,
                                                   int64_t idx) {
    if constexpr (FORM == kKahan32)
        return f32_to_f64(((const float *)u_main)[idx]) + f32_to_f64(((const float *)aux)[idx]);
    else if constexpr (FORM == kFP32Force)
        return join_state(((const float *)u_main)[idx], ((const uint32_t *)aux)[idx]);
    else
        return ((const double *)u_main)[idx];
}

template <int FORM>
__global__ void __launch_bounds__(256) stats_kernel(const void *__restrict__ u_main,
                                                    const void *__restrict__ aux, int32_t N,
                                                    int32_t S, int32_t Sp, double inv_s,
                                                    double inv_s1, double *__restrict__ mean,
                                                    double *__restrict__ var) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = t / kStatLanes;
    const int g = (int)(t % kStatLanes);
    const bool live = row < (int64_t)N * 3;
    const int64_t base = live ? row * Sp : 0;
    const bool in_regs = S <= kStatLanes * kStatRegs;
    double x[kStatRegs];
    double s = 0.0;
    if (live) {
        if (in_regs) {
#pragma unroll
            for (int k = 0; k < kStatRegs; k++) {
                const int32_t j = g + k * kStatLanes;
                x[k] = j < S ? state_value_fast<FORM>(u_main, aux, base + j) : 0.0;
                s += x[k];
            }
        } else {
            for (int32_t j = g; j < S; j += kStatLanes) s += state_value_fast<FORM>(u_main, aux, base + j);
        }
    }
#pragma unroll
    for (int o = kStatLanes / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double mu = s * inv_s;
    double q = 0.0;
    if (live) {
        if (in_regs) {
#pragma unroll
            for (int k = 0; k < kStatRegs; k++) {
                const int32_t j = g + k * kStatLanes;
                const double d = x[k] - mu;
                q = j < S ? fma(d, d, q) : q;
            }
        } else {
            for (int32_t j = g; j < S; j += kStatLanes) {
                const double d = state_value_fast<FORM>(u_main, aux, base + j) - mu;
                q = fma(d, d, q);
            }
        }
    }
#pragma unroll
    for (int o = kStatLanes / 2; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (live && g == 0) {
        mean[row] = mu;
        var[row] = q * inv_s1;
    }
}

template <int FORM>
__global__ void export_kernel(const void *__restrict__ u_main, const void *__restrict__ aux,
                              int32_t N, int32_t S, int32_t Sp, double *__restrict__ out,
                              int layout) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * 3 * S) return;
    const int64_t row = t / S;
    const int32_t s = (int32_t)(t - row * S);
    const double x = state_value_fast<FORM>(u_main, aux, row * Sp + s);
    if (layout == 0)
        out[(int64_t)s * N * 3 + row] = x;
    else
        out[t] = x;
}

// Load a binary64 [N][3][S] field into a gathered-precision buffer (force-only
// evaluations) as the form's state would hold it for the gather: binary64 as is; the
// FP32-force head, u truncated toward zero (magnitudes below 2^-126 as signed zero);
// the compensated form's hi part, u rounded to nearest. Padding samples are zero.
template <int FORM>
__global__ void import_kernel(const double *__restrict__ in, int32_t N, int32_t S, int32_t Sp,
                              void *ug) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * 3 * Sp) return;
    const int64_t row = t / Sp;
    const int32_t s = (int32_t)(t - row * Sp);
    const double x = s < S ? in[row * S + s] : 0.0;
    if constexpr (FORM == kFP64)
        ((double *)ug)[t] = x;
    else if constexpr (FORM == kFP32Force)
        ((float *)ug)[t] = f64_to_f32_rz(x);
    else
        ((float *)ug)[t] = (float)x;
}

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

thread_local char g_launch_note[160] = "";

void note_launch(const char *what, int block, int minb, uint32_t smem, cudaError_t e) {
    snprintf(g_launch_note, sizeof(g_launch_note), "%s (block %d, %d/SM, %u B shared): %s", what,
             block, minb, smem, cudaGetErrorString(e));
}

// Launch with programmatic stream serialisation: the kernel may begin while the previous
// kernel on the stream finishes (once every block of that kernel has signalled
// griddepcontrol.launch_dependents, or it has exited); the staged kernels then stage
// only their constant records before griddepcontrol.wait. Inside stream capture this
// becomes a programmatic dependency edge of the graph.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), unsigned grid, int block, uint32_t smem, cudaStream_t s,
                       Args &&...args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

template <int FORM, typename R, bool FO, int BLOCK, int MINB, int V = Vw<R>::V, bool HOIST = false,
          bool REC = false>
cudaError_t launch_staged(const StepArgs<R> &a0, cudaStream_t s, const StagePlan *plan) {
    auto *k = step_staged_kernel<FORM, R, FO, BLOCK, MINB, V, HOIST, REC>;
    StepArgs<R> a = a0;
    a.fv.Q = a.fv.Sp / V;
    if (plan->smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)plan->smem);
        if (e != cudaSuccess) {
            note_launch("cudaFuncSetAttribute", BLOCK, MINB, plan->smem, e);
            return e;
        }
    }
    const unsigned grid = (unsigned)((a.fv.N + plan->nb - 1) / plan->nb);
    cudaError_t e = launch_pdl(k, grid, BLOCK, plan->smem, s, a, *plan);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) note_launch("staged launch", BLOCK, MINB, plan->smem, e);
    return e;
}

template <int FORM, typename R, int BLOCK, int MINB, int V>
cudaError_t launch_pipelined(const StepArgs<R> &a0, cudaStream_t s, const StagePlan *plan) {
    auto *k = step_pipelined_kernel<FORM, R, BLOCK, MINB, V>;
    StepArgs<R> a = a0;
    a.fv.Q = a.fv.Sp / V;
    if (plan->smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan->smem);
        if (e != cudaSuccess) {
            note_launch("cudaFuncSetAttribute", BLOCK, MINB, plan->smem, e);
            return e;
        }
    }
    const int32_t n_tiles = (a.fv.N + plan->nb - 1) / plan->nb;
    int grid = plan->grid;
    if (grid <= 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, BLOCK, plan->smem);
        grid = sms * (per > 0 ? per : 1);
    }
    if (grid > n_tiles) grid = n_tiles;
    k<<<grid, BLOCK, plan->smem, s>>>(a, *plan, n_tiles);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) note_launch("pipelined launch", BLOCK, MINB, plan->smem, e);
    return e;
}

template <int FORM, typename R, bool FO>
cudaError_t launch_one(const StepArgs<R> &a, cudaStream_t s, const StagePlan *plan) {
    const int64_t threads = (int64_t)a.fv.N * a.fv.Q;
    if constexpr (!FO) {
        if (a.kcs) {  // geometry update: per-realisation blocks, one launch shape, two samples
                      // per thread (the per-incidence block loads need the registers)
            StepArgs<R> g = a;
            g.fv.Q = g.fv.Sp / 2;
            step_geom_kernel<FORM, R, 2><<<blocks_for((int64_t)g.fv.N * g.fv.Q, kBlock), kBlock, 0, s>>>(g);
            return cudaGetLastError();
        }
    }
    if (plan && plan->staged) {
        if constexpr (FO) {
            // force-only evaluations have one staged shape; other plans run unstaged
            if (plan->block == 256 && plan->minb == 4) return launch_staged<FORM, R, FO, 256, 4>(a, s, plan);
        } else {
            if constexpr (sizeof(R) == 4) {
                if (plan->pipelined) {
                    if (plan->block == 128) return launch_pipelined<FORM, R, 128, 8, 2>(a, s, plan);
                    return launch_pipelined<FORM, R, 256, 4, 2>(a, s, plan);
                }
                if (plan->rec) {
                    if (plan->vw == 2) return launch_staged<FORM, R, FO, 128, 10, 2, false, true>(a, s, plan);
                    if (plan->minb == 10) return launch_staged<FORM, R, FO, 64, 10, 4, false, true>(a, s, plan);
                    return launch_staged<FORM, R, FO, 64, 12, 4, false, true>(a, s, plan);
                }
                if (plan->vw == 2) {
                    if (plan->hoist) return launch_staged<FORM, R, FO, 128, 9, 2, true>(a, s, plan);
                    if (plan->block == 128) return launch_staged<FORM, R, FO, 128, 10, 2>(a, s, plan);
                    return launch_staged<FORM, R, FO, 256, 5, 2>(a, s, plan);
                }
            }
            if (plan->block == 128) return launch_staged<FORM, R, FO, 128, 6>(a, s, plan);
            if (plan->block == 64) return launch_staged<FORM, R, FO, 64, 12>(a, s, plan);
            if (plan->minb == 3) return launch_staged<FORM, R, FO, 256, 3>(a, s, plan);
            return launch_staged<FORM, R, FO, 256, 4>(a, s, plan);
        }
    }
    step_kernel<FORM, R, FO><<<blocks_for(threads, kBlock), kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

const char *last_launch_note() { return g_launch_note; }

template <typename R>
cudaError_t launch_step(int form, const StepArgs<R> &a, bool force_only, cudaStream_t s,
                        const StagePlan *plan) {
    if ((int64_t)a.fv.N * a.fv.Q == 0) return cudaSuccess;
    g_launch_note[0] = 0;
    if constexpr (sizeof(R) == 8) {
        return force_only ? launch_one<kFP64, double, true>(a, s, plan)
                          : launch_one<kFP64, double, false>(a, s, plan);
    } else {
        if (force_only) return launch_one<kKahan32, float, true>(a, s, plan);
        if (form == kFP32Force) return launch_one<kFP32Force, float, false>(a, s, plan);
        return launch_one<kKahan32, float, false>(a, s, plan);
    }
}

template <typename R>
cudaError_t launch_geo_correct(const StepArgs<R> &a0, const R *kcs_old, const R *kcs_new, double *c64, R *cR,
                               cudaStream_t s) {
    StepArgs<R> a = a0;
    a.fv.Q = a.fv.Sp / 2;  // two samples per thread, as the updated step
    const int64_t threads = (int64_t)a.fv.N * a.fv.Q;
    if (threads == 0) return cudaSuccess;
    geo_correct_kernel<R, 2><<<blocks_for(threads, kBlock), kBlock, 0, s>>>(a, kcs_old, kcs_new, c64, cR);
    return cudaGetLastError();
}
template cudaError_t launch_geo_correct<double>(const StepArgs<double> &, const double *, const double *, double *,
                                                double *, cudaStream_t);
template cudaError_t launch_geo_correct<float>(const StepArgs<float> &, const float *, const float *, double *,
                                               float *, cudaStream_t);

template cudaError_t launch_step<double>(int, const StepArgs<double> &, bool, cudaStream_t,
                                         const StagePlan *);
template cudaError_t launch_step<float>(int, const StepArgs<float> &, bool, cudaStream_t,
                                        const StagePlan *);

template <typename R>
cudaError_t launch_batch_step(int form, int block, const MemberDev<R> *mem, const int4 *items,
                              int32_t n_items, int32_t k_off, int *flags, cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    if constexpr (sizeof(R) == 8) {
        if (block == 128)
            batch_step_kernel<kFP64, double, 128><<<n_items, 128, 0, s>>>(mem, items, k_off, flags);
        else
            batch_step_kernel<kFP64, double, 256><<<n_items, 256, 0, s>>>(mem, items, k_off, flags);
    } else if (form == kFP32Force) {
        if (block == 128)
            batch_step_kernel<kFP32Force, float, 128><<<n_items, 128, 0, s>>>(mem, items, k_off, flags);
        else
            batch_step_kernel<kFP32Force, float, 256><<<n_items, 256, 0, s>>>(mem, items, k_off, flags);
    } else {
        if (block == 128)
            batch_step_kernel<kKahan32, float, 128><<<n_items, 128, 0, s>>>(mem, items, k_off, flags);
        else
            batch_step_kernel<kKahan32, float, 256><<<n_items, 256, 0, s>>>(mem, items, k_off, flags);
    }
    return cudaGetLastError();
}

template <int FORM, typename R, int BLOCK>
static cudaError_t coop_launch(const MemberDev<R> *mem, const int4 *items, int32_t n_items,
                               int32_t n_steps, unsigned *bar, int *flags, int grid, cudaStream_t s) {
    void *args[] = {(void *)&mem, (void *)&items, (void *)&n_items, (void *)&n_steps, (void *)&bar,
                    (void *)&flags};
    return cudaLaunchCooperativeKernel((const void *)batch_persistent_kernel<FORM, R, BLOCK>,
                                       dim3(grid), dim3(BLOCK), args, 0, s);
}

template <int FORM, typename R, int BLOCK>
static int coop_grid() {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_persistent_kernel<FORM, R, BLOCK>,
                                                      BLOCK, 0) != cudaSuccess)
        return 0;
    return sms * per;
}

template <typename R>
int batch_persistent_grid(int form, int block) {
    if constexpr (sizeof(R) == 8)
        return block == 128 ? coop_grid<kFP64, double, 128>() : coop_grid<kFP64, double, 256>();
    else if (form == kFP32Force)
        return block == 128 ? coop_grid<kFP32Force, float, 128>() : coop_grid<kFP32Force, float, 256>();
    else
        return block == 128 ? coop_grid<kKahan32, float, 128>() : coop_grid<kKahan32, float, 256>();
}

template <typename R>
cudaError_t launch_batch_persistent(int form, int block, const MemberDev<R> *mem,
                                    const int4 *items, int32_t n_items, int32_t n_steps,
                                    unsigned *bar, int *flags, int grid, cudaStream_t s) {
    if (n_items == 0 || n_steps == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if constexpr (sizeof(R) == 8) {
        return block == 128 ? coop_launch<kFP64, double, 128>(mem, items, n_items, n_steps, bar, flags, grid, s)
                            : coop_launch<kFP64, double, 256>(mem, items, n_items, n_steps, bar, flags, grid, s);
    } else if (form == kFP32Force) {
        return block == 128 ? coop_launch<kFP32Force, float, 128>(mem, items, n_items, n_steps, bar, flags, grid, s)
                            : coop_launch<kFP32Force, float, 256>(mem, items, n_items, n_steps, bar, flags, grid, s);
    } else {
        return block == 128 ? coop_launch<kKahan32, float, 128>(mem, items, n_items, n_steps, bar, flags, grid, s)
                            : coop_launch<kKahan32, float, 256>(mem, items, n_items, n_steps, bar, flags, grid, s);
    }
}

template cudaError_t launch_batch_step<double>(int, int, const MemberDev<double> *, const int4 *,
                                               int32_t, int32_t, int *, cudaStream_t);
template cudaError_t launch_batch_step<float>(int, int, const MemberDev<float> *, const int4 *,
                                              int32_t, int32_t, int *, cudaStream_t);
template cudaError_t launch_batch_persistent<double>(int, int, const MemberDev<double> *,
                                                     const int4 *, int32_t, int32_t, unsigned *,
                                                     int *, int, cudaStream_t);
template cudaError_t launch_batch_persistent<float>(int, int, const MemberDev<float> *,
                                                    const int4 *, int32_t, int32_t, unsigned *,
                                                    int *, int, cudaStream_t);
template int batch_persistent_grid<double>(int, int);
template int batch_persistent_grid<float>(int, int);

cudaError_t launch_advance_many(int64_t *const *ctrs, int32_t n, int64_t by, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    advance_many_kernel<<<(n + 127) / 128, 128, 0, s>>>(ctrs, n, by);
    return cudaGetLastError();
}

cudaError_t launch_fill(void *p, int64_t n, int is_double, float scale, uint32_t seed, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    fill_kernel<<<blocks_for(n, 256), 256, 0, s>>>(p, n, is_double, scale, seed);
    return cudaGetLastError();
}

cudaError_t launch_advance(int64_t *step_ctr, int64_t n, cudaStream_t s) {
    advance_kernel<<<1, 1, 0, s>>>(step_ctr, n);
    return cudaGetLastError();
}

cudaError_t launch_stats(int form, const void *u_main, const void *aux, int32_t N, int32_t S,
                         int32_t Sp, double *mean, double *var, cudaStream_t s) {
    const int64_t threads = (int64_t)N * 3 * kStatLanes;
    if (threads == 0) return cudaSuccess;
    const unsigned grid = blocks_for(threads, 256);
    const double inv_s = 1.0 / (double)S, inv_s1 = S > 1 ? 1.0 / (double)(S - 1) : 0.0;
    if (form == kKahan32)
        stats_kernel<kKahan32><<<grid, 256, 0, s>>>(u_main, aux, N, S, Sp, inv_s, inv_s1, mean, var);
    else if (form == kFP32Force)
        stats_kernel<kFP32Force><<<grid, 256, 0, s>>>(u_main, aux, N, S, Sp, inv_s, inv_s1, mean,
                                                      var);
    else
        stats_kernel<kFP64><<<grid, 256, 0, s>>>(u_main, aux, N, S, Sp, inv_s, inv_s1, mean, var);
    return cudaGetLastError();
}

cudaError_t launch_export(int form, const void *u_main, const void *aux, int32_t N, int32_t S,
                          int32_t Sp, double *out, int layout, cudaStream_t s) {
    const int64_t n = (int64_t)N * 3 * S;
    if (n == 0) return cudaSuccess;
    const unsigned grid = blocks_for(n, 256);
    if (form == kKahan32)
        export_kernel<kKahan32><<<grid, 256, 0, s>>>(u_main, aux, N, S, Sp, out, layout);
    else if (form == kFP32Force)
        export_kernel<kFP32Force><<<grid, 256, 0, s>>>(u_main, aux, N, S, Sp, out, layout);
    else
        export_kernel<kFP64><<<grid, 256, 0, s>>>(u_main, aux, N, S, Sp, out, layout);
    return cudaGetLastError();
}

cudaError_t launch_import(int form, const double *in_ncs, int32_t N, int32_t S, int32_t Sp,
                          void *ug, cudaStream_t s) {
    const int64_t n = (int64_t)N * 3 * Sp;
    if (n == 0) return cudaSuccess;
    const unsigned grid = blocks_for(n, 256);
    if (form == kFP64)
        import_kernel<kFP64><<<grid, 256, 0, s>>>(in_ncs, N, S, Sp, ug);
    else if (form == kFP32Force)
        import_kernel<kFP32Force><<<grid, 256, 0, s>>>(in_ncs, N, S, Sp, ug);
    else
        import_kernel<kKahan32><<<grid, 256, 0, s>>>(in_ncs, N, S, Sp, ug);
    return cudaGetLastError();
}

}  // namespace ens
