// Internal declarations shared by the library's translation units (not part of the ABI).
//
// Device data layout (sample index innermost, padded to Sp = round_up(S, 4) so every
// row of a per-sample array starts on a 16-byte boundary for float4 / double2 access):
//   u, v state            [N][3][Sp]     (precision-dependent, see StepArgs below)
//   per-element (E h)     [E][Sp]
//   inverse lumped mass   [N][Sp]
//   node -> element CSR   rowptr [N+1], ent [nnz] = {element, node a, node b, corner}
//                         where a, b are the element's other corners in cyclic order
//   coupling blocks       kc [nnz][KC]: the 3 x 3 blocks K_{c,a}, K_{c,b} (row-major) of
//                         the element matrix per unit E h, rows of the entry's corner c
//   traction patterns     [J][N][3], amplitudes [n_steps][J]
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ens {

constexpr int kBlock = 256;       // threads per block of the node kernels
constexpr int kMaxModes = 16;     // traction patterns per context

// Coupling-block storage per incidence: 18 values, padded to a 16-byte multiple.
template <typename R> struct Kc;
template <> struct Kc<double> { static constexpr int stride = 18; };  // 144 B
template <> struct Kc<float> { static constexpr int stride = 20; };   // 80 B

// Samples per thread: one 16-byte vector.
template <typename R> struct Vw;
template <> struct Vw<double> { static constexpr int V = 2; };
template <> struct Vw<float> { static constexpr int V = 4; };

enum Form : int { kFP64 = 0, kFP32Force = 1, kKahan32 = 2 };

// Everything the internal-force gather reads (shared by all forms).
template <typename R>
struct ForceView {
    const int32_t *rowptr;  // [N+1]
    const int4 *ent;        // [nnz]
    const R *kc;            // [nnz][Kc<R>::stride]
    const R *eh;            // [E][Sp]
    int32_t N, Sp, Q;       // Q = Sp / V threads per node
};

// Arguments of one step (or one force evaluation) for every form.
//   kFP64      : ug = u (double, ping-pong), v (double, in place)
//   kFP32Force : binary64 u stored bit-split: ug = its binary32 truncation (ping-pong),
//                utail = the 29 mantissa bits below it (in place); v64 binary64 (in place)
//   kKahan32   : ug = hi part of u (ping-pong), ulo (in place), v32 (in place)
template <typename R>
struct StepArgs {
    ForceView<R> fv;
    const R *ug_cur;  // gathered displacement at step n
    R *ug_next;       // written: displacement at step n + 1 (gather precision)
    uint32_t *utail;  // kFP32Force low mantissa bits of the binary64 state
    double *v64;      // kFP64 / kFP32Force velocity
    float *ulo;       // kKahan32 low part
    float *v32;       // kKahan32 velocity
    const R *minv;    // [N][Sp]
    const uint8_t *fix;  // [N] bit d set = dof d fixed
    const R *modes;   // [J][N][3]
    const R *amp;     // [n_amp][J]
    const int64_t *step_ctr;  // device step index of u_n at the start of the chunk
    int32_t k_off;    // this launch advances step (*step_ctr + k_off)
    int32_t J;
    double c1, c2, dt;  // v_new = c1 v + c2 a ; u_new = u + dt v_new
    float c1f, c2f, dtf;  // the same constants rounded to binary32 (binary32 forms)
    double *force_out;  // force-only mode: [N][3][Sp] binary64
    const R *kcs;       // geometry update: per-realisation corner blocks [E][3][9][Sp]
    const R *kcorr;     // geometry update: force correction f_int(u_m) - K_m u_m [N][3][Sp]
    int *flags;         // [0] bit 0: non-finite seen, bit 1: a bounded wait gave up
};

// Launch plan of the staged step kernel: each block owns `nb` consecutive nodes and
// bulk-copies their incidence entries, coupling blocks and own displacement rows into
// shared memory (cnt_max = most incidences of any block). staged = 0 selects the
// unstaged kernel (threads per node do not divide the block, or the plan exceeds smem).
struct StagePlan {
    int32_t staged;
    int32_t block;    // threads per block (256, 128 or 64)
    int32_t nb;       // nodes per block
    int32_t cnt_max;  // most incidences of any block
    uint32_t smem;    // dynamic shared memory per block
    int32_t minb;     // resident blocks per SM the register budget targets
    int32_t vw;       // samples per thread (the binary32 forms also have a 2-sample shape)
    int32_t hoist;    // issue the traction loads before the force loop
    int32_t pipelined;  // persistent CTAs with a double-buffered staging ring
    uint32_t stage;     // bytes of one staging buffer (pipelined plans)
    int32_t grid;       // CTAs of a pipelined launch (0: computed at first launch)
    // Fixed-stride block records (rec = 1): block b's incidence entries sit at
    // rec_ent + b (rec_h + cnt_max), after rec_h 16-byte words of block-local row offsets
    // (nb + 1 int32), and its coupling blocks at rec_kc + b cnt_max Kc<R>::stride, both
    // zero-padded to cnt_max entries. The block can then issue its bulk copies before any
    // global load, since every address and size follows from its index.
    int32_t rec;
    int32_t rec_h;
    const int4 *rec_ent;
    const void *rec_kc;
};

// One member of a batched launch (several contexts advanced by one kernel per step or
// by one persistent kernel). Built on the host before every batched call.
template <typename R>
struct MemberDev {
    ForceView<R> fv;
    const R *ug[2];         // ping-pong gathered displacement buffers
    uint32_t *utail;
    double *v64;
    float *ulo, *v32;
    const R *minv;
    const uint8_t *fix;
    const R *modes, *amp;
    int64_t *step_ctr;
    int32_t J;
    int32_t cur;            // buffer holding u_n at the start of the call
    int32_t first;          // the call's first step applies the start constants
    int32_t pad;
    double c1, c2, dt;      // regular update constants
    double c1s, c2s;        // start-step constants
};

// Spin iterations (each with a short sleep) of a grid-barrier wait before giving up.
constexpr uint32_t kSpinLimit = 1u << 24;

// Polls of a bounded mbarrier wait before the kernel reports a timeout.
constexpr uint32_t kWaitLimit = 1u << 22;

// Launchers (ens_step.cu).
template <typename R>
cudaError_t launch_step(int form, const StepArgs<R> &a, bool force_only, cudaStream_t s,
                        const StagePlan *plan = nullptr);

const char *last_launch_note();  // detail of this thread's last failed staged launch
// Batched launches (ens_step.cu). items: {member, first node, first lane, 0} tiles.
template <typename R>
cudaError_t launch_batch_step(int form, int block, const MemberDev<R> *mem, const int4 *items,
                              int32_t n_items, int32_t k_off, int *flags, cudaStream_t s);
template <typename R>
cudaError_t launch_batch_persistent(int form, int block, const MemberDev<R> *mem,
                                    const int4 *items, int32_t n_items, int32_t n_steps,
                                    unsigned *bar, int *flags, int grid, cudaStream_t s);
template <typename R>
int batch_persistent_grid(int form, int block);  // co-resident blocks of the persistent kernel
cudaError_t launch_advance_many(int64_t *const *ctrs, int32_t n, int64_t by, cudaStream_t s);
cudaError_t launch_advance(int64_t *step_ctr, int64_t n, cudaStream_t s);
cudaError_t launch_fill(void *p, int64_t n, int is_double, float scale, uint32_t seed, cudaStream_t s);
// u_main: the state's gathered buffer (binary64 u for the FP64 form); aux: the compensated
// form's low parts or the FP32-force form's tails (unused for FP64).
cudaError_t launch_stats(int form, const void *u_main, const void *aux, int32_t N, int32_t S,
                         int32_t Sp, double *mean, double *var, cudaStream_t s);
cudaError_t launch_export(int form, const void *u_main, const void *aux, int32_t N, int32_t S,
                          int32_t Sp, double *out, int layout, cudaStream_t s);
cudaError_t launch_import(int form, const double *in_ncs, int32_t N, int32_t S, int32_t Sp,
                          void *ug, cudaStream_t s);
// Geometry update: c64 += K_old u - K_new u per realisation (the internal forces of the
// state a.ug_cur under the old blocks, per-realisation kcs_old or the shared ones when
// null, and the new per-realisation blocks kcs_new), cR = c64 rounded to the force
// precision.
template <typename R>
cudaError_t launch_geo_correct(const StepArgs<R> &a, const R *kcs_old, const R *kcs_new, double *c64, R *cR,
                               cudaStream_t s);

// Setup launchers (ens_setup.cu).
cudaError_t launch_setup_elements(const double *xyz, const int32_t *tri, const int32_t *ec2ent,
                                  int32_t E, double nu, double kshear, double *kc64,
                                  double *area, double *lam_lo, double *lam_hi, double *xsq,
                                  double *kfull, int *bad, cudaStream_t s);
cudaError_t launch_setup_eh(const int32_t *tri, const double *E_node, const double *h_node,
                            int32_t E, int32_t Sp, double *eh64, cudaStream_t s);
cudaError_t launch_setup_mass(const int32_t *rowptr, const int4 *ent, const double *area,
                              const double *h_node, int32_t N, int32_t Sp, double rho,
                              double *m64, cudaStream_t s);
cudaError_t launch_setup_stability(const int32_t *tri, const double *eh64, const double *m64,
                                   const double *area, const double *h_node,
                                   const double *lam_lo, const double *lam_hi,
                                   const double *xsq, int32_t E, int32_t S, int32_t Sp,
                                   double rho, const double *rhoh, double *w2lo, double *w2hi,
                                   cudaStream_t s);
// Per-element coefficients (ENS_FLAG_ELEMENT_COEFFS): lumped mass from (rho hbar) [E][Sp],
// and the element modulus (E h) rho / (rho hbar) for the stress output.
cudaError_t launch_setup_mass_elem(const int32_t *rowptr, const int4 *ent, const double *area,
                                   const double *rhoh, int32_t N, int32_t Sp, double *m64, cudaStream_t s);
cudaError_t launch_modulus_from_coeffs(const double *eh64, const double *rhoh, int64_t n, double rho,
                                       double *ebar, cudaStream_t s);
// Geometry update (ens_setup.cu): per-realisation corner blocks kcs [E][3][9][Sp] (K_01,
// K_12, K_20 of each element) of the deformed surface xyz + u (u the state of the given
// form); bit 3 of *flags for an element that degenerated.
cudaError_t launch_reassemble(int form, const double *xyz, const int32_t *tri, int32_t E, int32_t Sp, double nu,
                              double kshear, const void *u_main, const void *aux, void *kcs, int *flags,
                              cudaStream_t s);
cudaError_t launch_pack_kc(const double *kc64, int64_t nnz, void *kc_out, int to_float,
                           cudaStream_t s);
// Binary32 coupling blocks (stride 20) into fixed-stride block records of nb nodes and
// cnt_max entries each (StagePlan::rec_kc), zero-padded.
cudaError_t launch_pack_records(const float *kc, const int32_t *rowptr, int32_t N, int32_t nb,
                                int32_t cnt_max, float *kc_rec, cudaStream_t s);
// Output statistics (ens_outputs.cu).
cudaError_t launch_element_mean(const int32_t *tri, const double *En, int32_t E, int32_t Sp, double *ebar,
                                cudaStream_t s);
cudaError_t launch_row_stats(const double *rows, int64_t n_rows, int32_t S, int32_t n_q, const double *q_dev,
                             double *mean, double *var, double *quant, cudaStream_t s);
// Running peak of |u| (ens_outputs.cu), kept squared: after the step launch k_off of a
// chunk whose first state index is *step_ctr, peak2 = max(peak2, |u|^2) when the new
// index is a multiple of stride; u_main: the gathered state words written by that launch
// (aux unused).
cudaError_t launch_peak(int form, const void *u_main, const void *aux, int32_t N, int32_t Sp,
                        const int64_t *step_ctr, int32_t k_off, int32_t stride, double *peak, cudaStream_t s);
cudaError_t launch_pad_fields(const double *src, int32_t N, int32_t S, int32_t Sp, double *dst,
                              int *bad, cudaStream_t s);
cudaError_t launch_convert(const double *in, int64_t n, void *out, int to_float, int invert,
                           cudaStream_t s);

}  // namespace ens
