/*
 * ens.h — C ABI of the GB300 explicit ensemble solver for the segregated vessel-wall
 * model of Li & Schiavazzi, "An ensemble solver for segregated cardiovascular FSI"
 * (arXiv 2101.09059).
 *
 * What is solved (Section 2.2.1 and Section 2.3, Eq. dynamicsCD): a small-strain,
 * linear, 3-dof-per-node shell of linear triangles (membrane plus transverse shear),
 * lumped mass M and mass-proportional damping C = alpha M, advanced by central
 * differences
 *     (M + dt/2 C) u_{n+1} = dt^2 f_n - (dt^2 K - 2 M) u_n - (M - dt/2 C) u_{n-1}
 * for S realisations at once. Each realisation s has its own nodal elastic modulus E_s
 * and thickness h_s (Section 2.1 random fields); every realisation sees the same wall
 * traction history f_n (one-way coupling, Section 2.2.3). The library evaluates the
 * equivalent velocity form v_{n+1/2} = ((1 - beta) v_{n-1/2} + dt a_n) / (1 + beta),
 * u_{n+1} = u_n + dt v_{n+1/2}, beta = alpha dt / 2, a_n = M^-1 (f_n - K_s u_n), with
 * K_s never stored (assembly-free, Section 2.4).
 *
 * Conventions shared by every entry point:
 *  - Units are the caller's; the shipped workloads use SI.
 *  - Every call returns ENS_OK (0) or a negative ENS_ERR_* code; ens_last_error gives
 *    the message of the last failing call on that context. No C++ exception crosses
 *    the ABI.
 *  - Host input arrays belong to the caller and are copied before the call returns.
 *    Output arrays are caller-allocated.
 *  - Device work runs on the stream given at creation. Calls that return host data
 *    synchronise that stream; ens_step synchronises it once at the end to report
 *    non-finite values. Long ens_step calls replay a CUDA graph of 32 step launches
 *    (captured on a private stream on first use), so the first such call must not be
 *    made while the context's stream is being captured.
 *  - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef ENS_H
#define ENS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------- */
#define ENS_OK 0
#define ENS_ERR_INVALID_ARG (-1) /* bad pointer, size, layout or parameter            */
#define ENS_ERR_ALLOC (-2)       /* device allocation failed                           */
#define ENS_ERR_CUDA (-3)        /* a CUDA runtime call failed (message has the name)  */
#define ENS_ERR_UNSTABLE_DT (-4) /* dt is above the central-difference stability limit */
#define ENS_ERR_NONFINITE (-5)   /* a displacement became Inf or NaN (FP32-force: left
                                    the binary32 range)                                 */
#define ENS_ERR_TIMEOUT (-6)     /* a bounded device-side wait gave up                 */
#define ENS_ERR_RANGE (-7)       /* stepping past the end of the traction table        */
#define ENS_ERR_STATE (-8)       /* call not valid in the current state                */

/* ---- precision forms ------------------------------------------------------------
 * ENS_FP64       : every operation in IEEE binary64.
 * ENS_FP32_FORCE : element forces K_s u in binary32 from u truncated to binary32; the
 *                  displacement and velocity state and their update stay binary64. The
 *                  displacement is stored bit-split (its binary32 truncation, which the
 *                  forces read, and the 29 mantissa bits below it), exact for magnitudes
 *                  in [2^-126, 2^128); smaller magnitudes are held as zero and larger ones
 *                  end the run with ENS_ERR_NONFINITE.
 * ENS_KAHAN32    : forces in binary32; the displacement is a compensated pair of
 *                  binary32 values (hi + lo) updated with an error-free sum, the
 *                  velocity is binary32.                                              */
typedef enum { ENS_FP64 = 0, ENS_FP32_FORCE = 1, ENS_KAHAN32 = 2 } ens_precision;

/* ---- creation flags (ens_params.flags) -------------------------------------------
 * ENS_FLAG_NO_AUTOTUNE : keep the default launch shape instead of timing candidates.
 * ENS_FLAG_UNSTAGED    : use the kernel without shared-memory staging.              */
#define ENS_FLAG_NO_AUTOTUNE 1
#define ENS_FLAG_UNSTAGED 2
/* Launch every step directly instead of replaying the captured time-loop graph (by
 * default ens_step replays a graph of 32 step launches when n allows).                */
#define ENS_FLAG_NO_GRAPH 4
/* Use launch shape k of ens_info_t.kernel_variant (when it applies to the context's
 * sizes; otherwise the unstaged kernel) instead of timing candidates.                 */
#define ENS_FLAG_FORCE_VARIANT(k) (((k) + 1) << 8)
/* E_node and h_node of ens_create are device pointers (binary64 [n_nodes][S] on the
 * context's device, e.g. written by gmrf_sample) instead of host pointers; they are
 * checked on the device (every value finite and > 0) and copied.                     */
#define ENS_FLAG_DEVICE_FIELDS 16
/* The two field arguments of ens_create are per-element coefficients instead of nodal
 * fields: E_node is read as eh host [n_elems][S], the Gauss-weighted product
 * (E h)_e,s = sum_gp w_gp E(gp) h(gp) of Section 2.2.1, and h_node as rho_h host
 * [n_elems][S], rho times the element's mean thickness, so that the lumped mass is
 * m_i,s = sum over elements of A_e rho_h_e,s / 3 (Section 2.3); params.rho is then used
 * only by the stress output, whose element modulus becomes E_e,s = eh_e,s rho / rho_h_e,s
 * (exact when E and h are constant on each element). Every value finite and > 0. Not
 * combinable with ENS_FLAG_DEVICE_FIELDS.                                             */
#define ENS_FLAG_ELEMENT_COEFFS 32

/* ---- displacement layouts for the getters ---------------------------------------- */
#define ENS_LAYOUT_SNC 0 /* out[s][node][dof]  */
#define ENS_LAYOUT_NCS 1 /* out[node][dof][s]  */

typedef struct ens_ctx ens_ctx;

/* Surface mesh of linear triangles (Section 2.2.1). Corner order fixes the outward
 * normal (X2 - X1) x (X3 - X1). fixed: per dof, 1 = held at zero ("fully fixed"
 * restraints of Section 3); NULL means nothing is fixed. Node ids in tri must be in
 * [0, n_nodes). Elements of zero area are rejected with ENS_ERR_INVALID_ARG.        */
typedef struct {
    int32_t n_nodes;
    int32_t n_elems;
    const double *xyz;    /* host [n_nodes][3]            */
    const int32_t *tri;   /* host [n_elems][3]            */
    const uint8_t *fixed; /* host [n_nodes][3] or NULL    */
} ens_mesh;

/* Material and integration constants.
 * rho    : density (lumped mass m_i = sum over elements of rho A_e hbar_e / 3).
 * nu     : Poisson ratio of the constitutive matrix C (Section 2.2.1), 0 <= nu < 1.
 * kshear : transverse shear factor k (5/6 in the paper).
 * alpha  : mass-proportional damping C = alpha M, >= 0.
 * dt     : time step, > 0. ens_create returns ENS_ERR_UNSTABLE_DT when dt exceeds
 *          2 / omega_lower, where omega_lower^2 is an element-local Rayleigh quotient
 *          of M^-1 K_s (a lower bound of the top eigenvalue, so such a dt certainly
 *          diverges). omega_upper (element eigenvalue bound) is reported by ens_info:
 *          dt <= 2 / omega_upper is guaranteed stable.
 * precision : an ens_precision value. flags : ENS_FLAG_* bits (0 = default: the
 *          launch shape of the step kernel is chosen by timing a few candidate shapes
 *          on the context's own data at rest during ens_create).                      */
typedef struct {
    double rho;
    double nu;
    double kshear;
    double alpha;
    double dt;
    int32_t precision;
    int32_t flags;
} ens_params;

/* Optional device allocator. alloc returns a device pointer of at least `bytes`
 * bytes (aligned to 256 bytes) usable on `stream`, or NULL on failure; release frees
 * it. NULL allocator: cudaMalloc / cudaFree.                                        */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*release)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} ens_allocator;

/* Sizes and the traffic model of one context (read-only report).                    */
typedef struct {
    int32_t n_nodes, n_elems, n_samples, n_samples_padded;
    int32_t precision, n_modes;
    int64_t n_steps_table; /* rows of the traction amplitude table              */
    int64_t step;          /* index n of the current state u_n                  */
    int64_t nnz;           /* node-to-element incidences (3 n_elems)            */
    double dt;
    double omega_lower;     /* lower bound of the top angular frequency         */
    double omega_upper;     /* upper bound of the top angular frequency         */
    double bytes_per_step;  /* algorithmic HBM bytes of one step                */
    double device_bytes;    /* device memory held by the context                */
    int32_t kernel_variant; /* launch shape in use: 0 unstaged, 1 staged 256x4,
                               2 staged 256x3, 3 staged 128x6, 4 staged 64x12
                               (threads per block x blocks per SM), 5 staged 256x5
                               and 6 staged 128x10 with two samples per thread
                               (binary32 forms), 7 staged 128x9 with two samples
                               per thread and the traction loads issued before
                               the force loop, 8 and 9 persistent double-buffered
                               forms of 5 and 6, 10 and 11 the shapes of 6 and 4
                               staged from fixed-stride block records (binary32
                               forms), 12 shape 11 at 10 blocks per SM (more
                               registers per thread)                              */
    float variant_us[16];   /* autotuner's time per step of shapes 0..12 (-1: n/a,
                               0: not timed; entries 13..15 unused)               */
} ens_info_t;

/* Create a context: copies the mesh, builds the node-to-element incidence lists,
 * computes on the device the element matrices per unit E*h (Section 2.2.1: B, C,
 * k_e = sum_gp B^T C B A_e zeta w), the three-point Gauss products (E*h)_e,s and the
 * lumped masses (Section 2.3), and sets the state to rest (u_0 = v_0 = 0).
 * S       : ensemble width, >= 1.
 * E_node, h_node : host [n_nodes][S] nodal modulus and thickness of every
 *           realisation (sample index innermost), all > 0 (device arrays with
 *           ENS_FLAG_DEVICE_FIELDS; per-element eh and rho_h [n_elems][S] with
 *           ENS_FLAG_ELEMENT_COEFFS).
 * stream  : cudaStream_t to run on (NULL = legacy default stream).
 * alloc   : device allocator or NULL.
 * out     : receives the context; on failure *out is NULL and the code is returned
 *           (use ens_error_string for the text).                                   */
int ens_create(const ens_mesh *mesh, int32_t S, const double *E_node, const double *h_node,
               const ens_params *params, void *stream, const ens_allocator *alloc,
               ens_ctx **out);

/* Wall traction history in separable form f_n = sum_j amp[n][j] * modes[j]
 * (Section 2.2.3: the nodal force passed from the fluid to the structure; identical
 * for every realisation). modes: host [J][n_nodes][3]; amp: host [n_steps][J].
 * 1 <= J <= 16. All values finite (and within the binary32 range for the binary32
 * forms). Replaces any previous table; the state is kept.                            */
int ens_set_traction(ens_ctx *ctx, int32_t J, const double *modes, int64_t n_steps,
                     const double *amp);

/* Overwrite rows [first_row, first_row + n_rows) of the current amplitude table with
 * amp (host [n_rows][J], J of the last ens_set_traction): the way a coupled fluid
 * solver streams new load amplitudes while the structure advances (Section 2.2.3).
 * The copy is ordered on the context stream before later steps; the host buffer may
 * be reused when the call returns. ENS_ERR_RANGE if the rows fall outside the table. */
int ens_set_amplitudes(ens_ctx *ctx, int64_t first_row, int64_t n_rows, const double *amp);

/* Advance every realisation n >= 0 steps of Eq. (dynamicsCD) from the current step
 * index; step k uses load row amp[k]. The first step after creation or ens_reset
 * applies the Taylor start u_{-1} = u_0 - dt v_0 + dt^2/2 a_0. Returns ENS_ERR_RANGE
 * (nothing is run) if the table has fewer than index + n rows, ENS_ERR_NONFINITE if a
 * displacement became Inf/NaN during these steps.                                    */
int ens_step(ens_ctx *ctx, int64_t n);

/* Back to rest: u = v = 0, step index 0 (with a geometry update, the per-realisation
 * stiffness is re-assembled on the reference surface).                               */
int ens_reset(ens_ctx *ctx);

/* Geometry update with selective stiffness re-assembly (Section 2.3: the system
 * M u'' + C u' + K(u) u = f, the lumen geometry updated by the displacement at every
 * step, the stiffness re-assembled only after a prescribed number of iterations, the
 * lumped mass and the traction history kept fixed). K(u) is the stiffness of the current
 * surface applied to displacement increments: with k >= 1, at every step index m that is
 * a multiple of k (after this call) each realisation's coupling blocks are re-assembled
 * on its deformed surface X + u_s,m (scaled by the same (E h)_e,s), and the steps from m
 * use f_int(u_n) = f_int(u_m) + K(X + u_m) (u_n - u_m). Before the first re-assembly the
 * run is the linear method (bit for bit). k = 0 returns to the linear method and frees
 * the per-realisation data: two block buffers of E * 27 * Sp values (the element
 * matrix's three corner blocks K_01, K_12, K_20, the others being their transposes) in
 * the form's force precision (binary64 for ENS_FP64, binary32 otherwise) and the force correction
 * f_int(u_m) - K_m u_m, N * 3 * Sp values in binary64 plus its force-precision copy.
 * ens_reset and ens_set_state return to the linear stiffness with a zero correction (the
 * checkpoint holds neither); ens_internal_force keeps the reference blocks. A step with
 * per-realisation blocks streams them (108 B per element and sample in binary32, each
 * block read by the two corners it couples) instead of the shared ones, several times
 * the bytes of a linear step; a re-assembly
 * costs one binary64 pass over the elements and samples (the new blocks) and one over the
 * nodes and samples, which adds (K_old - K_new) u_m to the correction: coefficient
 * differences first, in the form's precision, the running sum in binary64, so the binary32
 * forms' rounding of full forces does not accumulate in it.
 * Selective re-assembly (k > 1) uses the stiffness of a segment's start for the whole
 * segment, a path error of order k. An element that degenerates on its deformed surface
 * ends ens_step with ENS_ERR_NONFINITE. Contexts with a geometry update cannot join a
 * batch.                                                                              */
int ens_set_geometry_update(ens_ctx *ctx, int32_t k);

/* Current displacements u_n as binary64. out: host array of S * n_nodes * 3 values in
 * the given ENS_LAYOUT_*.                                                             */
int ens_get_displacement(ens_ctx *ctx, double *out, int32_t layout);

/* Same into device memory (binary64, caller-allocated, same sizes and layouts).      */
int ens_get_displacement_device(ens_ctx *ctx, double *out_dev, int32_t layout);

/* Ensemble mean and sample variance (divisor S - 1, 0 when S = 1) of u_n per dof
 * (the ensemble means and bands of Section 3). mean, var: host [n_nodes][3].         */
int ens_stats(ens_ctx *ctx, double *mean, double *var);

/* Same into device memory (binary64 [n_nodes][3] each); runs asynchronously.        */
int ens_stats_device(ens_ctx *ctx, double *mean_dev, double *var_dev);

/* Internal force K_s u_s of every realisation for a given displacement field
 * (Section 2.4 assembly-free product; the term dt^2 K u_n of Eq. dynamicsCD without
 * dt^2), computed by the same device path and precision as ens_step. u is first brought
 * to the value the form's step gathers: binary64 as is (ENS_FP64), truncated toward
 * zero to binary32 (ENS_FP32_FORCE, the state's head), rounded to nearest binary32
 * (ENS_KAHAN32, the state's hi part). For a u that a state of the context holds, f is
 * bit for bit the internal force the next step applies. u, f: host [n_nodes][3][S]
 * binary64; u finite, and below 2^128 in magnitude for the binary32 forms
 * (ENS_ERR_INVALID_ARG otherwise). The context state is not changed.               */
int ens_internal_force(ens_ctx *ctx, const double *u, double *f);

/* The same internal force as ens_internal_force, for callers that may not allocate
 * device memory at this point (a host framework that owns all device memory, or a
 * loop where cudaMalloc and its implicit synchronisation are not allowed). The paper
 * has no counterpart; this is a library service.
 * u_dev, f_dev: device [n_nodes][3][S] binary64, caller-owned, on the context's device.
 * Staging lives in one static device array of 32 MiB per GPU (held from library load
 * to process exit); contexts needing more than n_nodes * 3 * Sp * (e + 8) <= 32 MiB
 * (e = 8 for ENS_FP64, 4 otherwise) get ENS_ERR_INVALID_ARG. Nothing is allocated.
 * The first call on a device looks the array's address up (cudaGetSymbolAddress); make
 * that first call before any stream capture. Asynchronous on the context stream. All
 * calls share the one array, so calls that overlap on the GPU (other streams, other
 * contexts on the same device) race; every staged value is rewritten before it is read,
 * so a call never sees the previous call's contents. Unlike ens_internal_force, which
 * reads u on the host and rejects non-finite values, this call does not inspect u_dev:
 * an Inf or NaN in u_dev gives non-finite forces in f_dev and no error code.          */
int ens_internal_force_noalloc(ens_ctx *ctx, const double *u_dev, double *f_dev);

/* Per-realisation coefficients as binary64 (Section 2.2.1 Gauss rule, Section 2.3
 * lumped mass): eh host [n_elems][S] = sum_gp w E zeta, minv host [n_nodes][S] =
 * 1 / m. Either pointer may be NULL.                                                 */
int ens_get_coefficients(ens_ctx *ctx, double *eh, double *minv);

/* Element matrices per unit E*h in the global frame (Section 2.2.1), binary64, as the
 * device computed them: kelem host [n_elems][9][9].                                  */
int ens_get_element_matrices(ens_ctx *ctx, double *kelem);

/* Checkpoint. ens_state_size gives the byte size; ens_get_state writes the state
 * (step index, start flag, u, v in the context's precision) to a host buffer;
 * ens_set_state restores one written by a context of identical sizes and precision. */
int ens_state_size(const ens_ctx *ctx, size_t *bytes);
int ens_get_state(ens_ctx *ctx, void *buf, size_t bytes);
int ens_set_state(ens_ctx *ctx, const void *buf, size_t bytes);

/* ---- batched launches --------------------------------------------------------------
 * Several contexts (different meshes, ensemble widths, time steps and traction tables;
 * one precision form, one device) advanced together. This is not in the paper, whose
 * ensembles share one mesh; it serves campaigns over uneven models.
 * Modes: ENS_BATCH_GRAPH runs one kernel per step covering every member, with the time
 * loop captured in a CUDA graph of 20-step chunks; ENS_BATCH_PERSISTENT runs all steps
 * of a call in one cooperative kernel with a grid barrier between steps (bounded wait:
 * ENS_ERR_TIMEOUT if it gives up); ENS_BATCH_SEQUENCE runs every member's own tuned
 * step kernel back to back per step, the loop captured in a graph; ENS_BATCH_AUTO times
 * every mode and block shape on the members' own data during ens_batch_create (states
 * are restored) and keeps the fastest.                                                */
#define ENS_BATCH_AUTO 0
#define ENS_BATCH_GRAPH 1
#define ENS_BATCH_PERSISTENT 2
#define ENS_BATCH_SEQUENCE 3

typedef struct ens_batch ens_batch;

typedef struct {
    int32_t n_members;
    int32_t mode;            /* ENS_BATCH_GRAPH, _PERSISTENT or _SEQUENCE in use    */
    int32_t block;           /* threads per block (256 or 128; 0: members' own)     */
    int32_t graph_steps;     /* steps per captured graph                            */
    int32_t n_tiles;         /* work tiles per step (about 1024 node-samples each)  */
    int32_t persistent_grid; /* co-resident blocks of the persistent kernel         */
    float mode_us[5];        /* autotuner time per step: graph 256, graph 128,
                                persistent 256, persistent 128, sequence
                                (-1: not possible, 0: not timed)                    */
    double bytes_per_step;   /* algorithmic HBM bytes of one batched step           */
} ens_batch_info_t;

/* Create a batch over n >= 1 distinct contexts (not owned; destroy the batch first).
 * mode: ENS_BATCH_*. Errors: ENS_ERR_INVALID_ARG (mixed forms or devices, repeated
 * members); the message is left on members[0] (ens_last_error).                        */
int ens_batch_create(ens_ctx *const *members, int32_t n, int32_t mode, ens_batch **out);

/* Advance every member n >= 0 steps (each with its own dt and load rows), exactly as n
 * calls of ens_step on each member would. Ordered after every member's pending work;
 * returns after the work completes. ENS_ERR_RANGE / ENS_ERR_STATE as ens_step.        */
int ens_batch_step(ens_batch *b, int64_t n);

int ens_batch_info(const ens_batch *b, ens_batch_info_t *info);
const char *ens_batch_last_error(const ens_batch *b);
void ens_batch_destroy(ens_batch *b);

/* Merge per-dof ensemble statistics of disjoint sample shards (e.g. one per GPU, each
 * from ens_stats): counts[k] samples with mean means[k][i] and sample variance vars[k][i]
 * (divisor counts[k] - 1) give the statistics of the union, mean_out[i] and var_out[i]
 * (divisor total - 1), for i < n. Host arrays; no device work. The mean is merged first
 * and the squared deviations are then summed around it (Chan et al.'s parallel form).
 * The paper's ensemble means and bands (Section 3) are of one ensemble; the merge lets
 * the realisations of one ensemble live on several GPUs with no exchange until here.   */
int ens_merge_stats(int32_t n_parts, const int64_t *counts, const double *const *means,
                    const double *const *vars, int64_t n, double *mean_out, double *var_out);

/* ---- output statistics (Section 3: mean displacement magnitude with 5 %-95 % bands,
 * displacement and stress time histories at chosen locations, stress in the local
 * cylindrical frame) ----------------------------------------------------------------
 * A quantity is a set of rows, each with one binary64 value per realisation, formed on
 * the device from the current state of any precision form:
 *   ENS_QTY_DISPLACEMENT    rows (node, dof)        n_nodes * 3 rows
 *   ENS_QTY_DISP_MAGNITUDE  rows node, |u|          n_nodes rows
 *   ENS_QTY_STRESS          rows (element, k)       n_elems * 6 rows, k = rr, tt, zz, rt, rz, tz
 * Stress follows Section 2.2.1 and the frame of Section 2.2.3: sigma_l = C(E) B u_l in the
 * element frame with E the element mean of the nodal modulus (the average of the linear
 * field over the three Gauss points), the plane-stress tensor (sigma_nn = 0) expressed in
 * r = the element's outward normal, t = (r x a) / |r x a|, z = a projected on the wall and
 * normalised, where a is the tangent of the centreline segment closest to the element
 * centroid.                                                                           */
#define ENS_QTY_DISPLACEMENT 0
#define ENS_QTY_DISP_MAGNITUDE 1
#define ENS_QTY_STRESS 2
/* Running peak over time (needs ens_set_peak), rows node: n_nodes rows, the largest
 * |u_k| over the recorded steps k.                                                    */
#define ENS_QTY_PEAK_MAGNITUDE 3

/* Centreline polyline for the stress frame: pts host [n_pts][3], n_pts >= 2. Builds the
 * per-element stress operators on the device (6 x 9 binary64 values per element).
 * ENS_ERR_INVALID_ARG if an element's normal is parallel to its centreline tangent.    */
int ens_set_centerline(ens_ctx *ctx, int32_t n_pts, const double *pts);

/* Rows of a quantity at the current step: out device [rows][S] binary64 (sample index
 * innermost). Runs on the context stream (asynchronous). ENS_ERR_STATE for stress
 * without a centreline.                                                               */
int ens_quantity_device(ens_ctx *ctx, int32_t qty, double *out);

/* Per-row statistics of a quantity at the current step: mean [rows], sample variance
 * [rows] (divisor S - 1; 0 when S = 1) and quantiles quant [rows][n_q] of type 7:
 * with the row's samples sorted ascending x_0 <= ... <= x_{S-1}, h = q_k (S - 1),
 * j = floor(h), quant = x_j + (h - j) (x_{j+1} - x_j) (x_j itself when j = S - 1),
 * evaluated without fused multiply-adds. Host outputs; any of mean, var may be NULL;
 * quant may be NULL only when n_q = 0. q host [n_q], each in [0, 1]; n_q <= 1024;
 * S <= 16384. Synchronises the context stream.                                         */
int ens_quantity_stats(ens_ctx *ctx, int32_t qty, int32_t n_q, const double *q, double *mean,
                       double *var, double *quant);

/* The same statistics for caller rows: rows device [n_rows][S] binary64, outputs device
 * (mean [n_rows], var [n_rows], quant [n_rows][n_q]; mean and var may be NULL), q host.
 * No context; runs on stream and synchronises it. 1 <= S <= 16384.                     */
int ens_row_stats_device(int64_t n_rows, int32_t S, const double *rows, int32_t n_q,
                         const double *q, double *mean, double *var, double *quant,
                         void *stream);

/* Running peak of the displacement magnitude per node and realisation (the peak and
 * band quantities of Section 3 over a heart cycle): with stride >= 1, every step that
 * ends on an index k that is a multiple of stride updates peak = max(peak, |u_k|); read
 * it as ENS_QTY_PEAK_MAGNITUDE. |u| is formed in binary64 for ENS_FP64 and in binary32
 * from the displacement words the binary32 forms gather (the FP32-force head, the
 * compensated hi part: within one binary32 rounding of the state). The call zeroes the
 * peak (so it covers steps after the call), as does ens_reset; stride = 0 switches
 * tracking off and frees it. The peak is kept squared by a separate kernel after each
 * step launch (also inside the captured time-loop graphs): per recorded step it reads
 * the gathered state once (12 B per node and sample in binary32, 24 B in binary64) and
 * reads and writes the peak (16 B). It is not part of ens_get_state's checkpoint, and
 * contexts that track a peak cannot join a batch (ens_batch_create / ens_batch_step
 * return ENS_ERR_STATE).                                                              */
int ens_set_peak(ens_ctx *ctx, int32_t stride);

/* Probe time histories: after every ens_step segment that ends on a step index that is
 * a multiple of stride, record the displacement of n_nodes probe nodes (all dofs, all
 * samples) and the stress of n_elems probe elements (needs a centreline), up to
 * capacity records (further records are dropped). stride = 0 switches probes off and
 * drops the history; ens_reset empties it. ids host arrays, copied.                    */
int ens_set_probes(ens_ctx *ctx, int32_t n_nodes, const int32_t *nodes, int32_t n_elems,
                   const int32_t *elems, int32_t stride, int64_t capacity);

/* Copy the history: u_out host [n_rec][n_nodes][3][S], sigma_out host
 * [n_rec][n_elems][6][S] (either may be NULL), steps_out host [n_rec] (the step index of
 * each record, may be NULL); *n_rec receives the number of records.                    */
int ens_get_probes(ens_ctx *ctx, double *u_out, double *sigma_out, int64_t *steps_out,
                   int64_t *n_rec);

/* Sizes, step index and traffic model.                                               */
int ens_info(const ens_ctx *ctx, ens_info_t *info);

/* Message of the last failing call on ctx ("" if none); with ctx = NULL, the message
 * of the calling thread's last failed ens_create. ens_error_string names a code. Both
 * return static, thread-owned or context-owned storage.                               */
const char *ens_last_error(const ens_ctx *ctx);
const char *ens_error_string(int code);

/* Release every device and host resource of the context (NULL is a no-op).          */
void ens_destroy(ens_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* ENS_H */
