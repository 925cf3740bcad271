// One-time set-up kernels: element coupling blocks (Section 2.2.1), Gauss-point products
// and lumped masses (Section 2.2.1 three-point rule, Section 2.3 lumped M), and the
// element-local stability bounds of the central-difference step.
//
// Everything here runs once per context in binary64; the time loop never calls it.
#include "ens_bits.cuh"
#include "ens_internal.cuh"

namespace ens {

namespace {

__device__ __forceinline__ void cross(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Element matrix per unit (E h), written block by block in closed form.
//
// With the linear-triangle shape-function gradients dN_j/dx = beta_j / (2A) and
// dN_j/dy = gamma_j / (2A) in a local in-plane frame (beta = (y23, y31, y12),
// gamma = (x32, x13, x21), the entries of B in Section 2.2.1), the product
// A B^T C0 B couples corner c to corner k through a 3 x 3 block whose only non-zero
// local entries are
//   xx = (b_c b_k C11 + g_c g_k C33) / 4A     xy = (b_c g_k C12 + g_c b_k C33) / 4A
//   yx = (g_c b_k C12 + b_c g_k C33) / 4A     yy = (g_c g_k C11 + b_c b_k C33) / 4A
//   zz = (b_c b_k + g_c g_k) C44 / 4A
// (C0 = C / E: C11 = 1/(1-nu^2), C12 = nu C11, C33 = (1-nu)/2 C11, C44 = k (1-nu)/2 C11).
// The block is rotated to the global frame with the local axes (t1, t2, n):
//   G[p][q] = t1_p (xx t1_q + xy t2_q) + t2_p (yx t1_q + yy t2_q) + n_p zz n_q.
// The in-plane axis t1 is taken along edge 1 -> 3; the block does not depend on that
// choice (the membrane and shear energies are isotropic in the plane).
struct ElemFrame {
    double t1[3], t2[3], n[3];
    double b[3], g[3];
    double area;
};

// RECIP: scale by the reciprocals of |n| and |X_2 - X_0| (two binary64 divisions instead
// of six, results within a few ulp of the quotients); the set-up kernel divides.
template <bool RECIP = false>
__device__ __forceinline__ bool element_frame(const double X[3][3], ElemFrame &f) {
    double a[3], c[3], nn[3];
    for (int d = 0; d < 3; d++) {
        a[d] = X[1][d] - X[0][d];
        c[d] = X[2][d] - X[0][d];
    }
    cross(a, c, nn);
    double twoA = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
    double lc = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    if (!(twoA > 0.0) || !(lc > 0.0) || !isfinite(twoA)) return false;
    if constexpr (RECIP) {
        const double in = 1.0 / twoA, ic = 1.0 / lc;
        for (int d = 0; d < 3; d++) {
            f.n[d] = nn[d] * in;
            f.t1[d] = c[d] * ic;
        }
    } else {
        for (int d = 0; d < 3; d++) {
            f.n[d] = nn[d] / twoA;
            f.t1[d] = c[d] / lc;
        }
    }
    cross(f.n, f.t1, f.t2);
    double x[3], y[3];
    for (int j = 0; j < 3; j++) {
        double r[3] = {X[j][0] - X[0][0], X[j][1] - X[0][1], X[j][2] - X[0][2]};
        x[j] = r[0] * f.t1[0] + r[1] * f.t1[1] + r[2] * f.t1[2];
        y[j] = r[0] * f.t2[0] + r[1] * f.t2[1] + r[2] * f.t2[2];
    }
    f.b[0] = y[1] - y[2];
    f.b[1] = y[2] - y[0];
    f.b[2] = y[0] - y[1];
    f.g[0] = x[2] - x[1];
    f.g[1] = x[0] - x[2];
    f.g[2] = x[1] - x[0];
    f.area = 0.5 * twoA;
    return true;
}

__device__ __forceinline__ void coupling_block(const ElemFrame &f, int c, int k, double nu,
                                               double ks, double G[3][3]) {
    const double C11 = 1.0 / (1.0 - nu * nu);
    const double C12 = nu * C11;
    const double C33 = 0.5 * (1.0 - nu) * C11;
    const double C44 = 0.5 * ks * (1.0 - nu) * C11;
    const double s = 1.0 / (4.0 * f.area);
    const double bc = f.b[c], gc = f.g[c], bk = f.b[k], gk = f.g[k];
    const double xx = s * (bc * bk * C11 + gc * gk * C33);
    const double xy = s * (bc * gk * C12 + gc * bk * C33);
    const double yx = s * (gc * bk * C12 + bc * gk * C33);
    const double yy = s * (gc * gk * C11 + bc * bk * C33);
    const double zz = s * (bc * bk + gc * gk) * C44;
    for (int p = 0; p < 3; p++)
        for (int q = 0; q < 3; q++)
            G[p][q] = f.t1[p] * (xx * f.t1[q] + xy * f.t2[q]) +
                      f.t2[p] * (yx * f.t1[q] + yy * f.t2[q]) + f.n[p] * zz * f.n[q];
}

__global__ void setup_elements_kernel(const double *__restrict__ xyz,
                                      const int32_t *__restrict__ tri,
                                      const int32_t *__restrict__ ec2ent, int32_t E, double nu,
                                      double ks, double *__restrict__ kc64,
                                      double *__restrict__ area, double *__restrict__ lam_lo,
                                      double *__restrict__ lam_hi, double *__restrict__ xsq,
                                      double *__restrict__ kfull, int *__restrict__ bad) {
    int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    double X[3][3];
    for (int j = 0; j < 3; j++)
        for (int d = 0; d < 3; d++) X[j][d] = xyz[3 * (int64_t)tri[3 * e + j] + d];
    ElemFrame f;
    if (!element_frame(X, f)) {
        atomicMin(bad, e);
        area[e] = 0.0;
        return;
    }
    area[e] = f.area;
    double K[9][9];
    for (int c = 0; c < 3; c++)
        for (int k = 0; k < 3; k++) {
            double G[3][3];
            coupling_block(f, c, k, nu, ks, G);
            for (int p = 0; p < 3; p++)
                for (int q = 0; q < 3; q++) K[3 * c + p][3 * k + q] = G[p][q];
        }
    if (kc64 != nullptr) {
        for (int c = 0; c < 3; c++) {
            int64_t p = ec2ent[3 * e + c];
            double *dst = kc64 + 18 * p;
            int a = (c + 1) % 3, b = (c + 2) % 3;
            for (int r = 0; r < 3; r++)
                for (int q = 0; q < 3; q++) {
                    dst[3 * r + q] = K[3 * c + r][3 * a + q];
                    dst[9 + 3 * r + q] = K[3 * c + r][3 * b + q];
                }
        }
    }
    if (kfull != nullptr)
        for (int r = 0; r < 9; r++)
            for (int q = 0; q < 9; q++) kfull[81 * (int64_t)e + 9 * r + q] = K[r][q];
    if (lam_lo == nullptr) return;
    // Upper bound of the top eigenvalue: largest absolute row sum (Gershgorin).
    double gmax = 0.0;
    for (int r = 0; r < 9; r++) {
        double s = 0.0;
        for (int q = 0; q < 9; q++) s += fabs(K[r][q]);
        gmax = fmax(gmax, s);
    }
    // Lower bound: Rayleigh quotient after power iteration (any unit vector gives one).
    double x[9];
    for (int r = 0; r < 9; r++) x[r] = (r % 2 ? -1.0 : 1.0) * (1.0 + 0.1 * r);
    for (int it = 0; it < 80; it++) {
        double y[9], nrm = 0.0;
        for (int r = 0; r < 9; r++) {
            double s = 0.0;
            for (int q = 0; q < 9; q++) s += K[r][q] * x[q];
            y[r] = s;
            nrm += s * s;
        }
        nrm = sqrt(nrm);
        if (!(nrm > 0.0)) break;
        for (int r = 0; r < 9; r++) x[r] = y[r] / nrm;
    }
    double xx = 0.0, xkx = 0.0;
    for (int r = 0; r < 9; r++) {
        double s = 0.0;
        for (int q = 0; q < 9; q++) s += K[r][q] * x[q];
        xkx += x[r] * s;
        xx += x[r] * x[r];
    }
    lam_lo[e] = xx > 0.0 ? xkx / xx : 0.0;
    lam_hi[e] = gmax;
    for (int c = 0; c < 3; c++)
        xsq[3 * e + c] = (x[3 * c] * x[3 * c] + x[3 * c + 1] * x[3 * c + 1] +
                          x[3 * c + 2] * x[3 * c + 2]) / (xx > 0.0 ? xx : 1.0);
}

// The same block in binary32 arithmetic from a binary64 frame rounded to binary32: for the
// binary32 forms, whose blocks are stored in binary32. Against the binary64 block rounded
// to binary32 the entries differ by at most about 4e-7 of the block's largest entry (a
// sweep over 4,000 random triangles; the storage rounding alone is 6e-8).
__device__ __forceinline__ void coupling_block_f32(const float (&t1)[3], const float (&t2)[3], const float (&n)[3],
                                                   float bc, float gc, float bk, float gk, float s, float C11,
                                                   float C12, float C33, float C44, float G[3][3]) {
    const float xx = s * (bc * bk * C11 + gc * gk * C33);
    const float xy = s * (bc * gk * C12 + gc * bk * C33);
    const float yx = s * (gc * bk * C12 + bc * gk * C33);
    const float yy = s * (gc * gk * C11 + bc * bk * C33);
    const float zz = s * (bc * bk + gc * gk) * C44;
    for (int q = 0; q < 3; q++) {
        const float uq = xx * t1[q] + xy * t2[q], wq = yx * t1[q] + yy * t2[q], zq = zz * n[q];
        for (int p = 0; p < 3; p++) G[p][q] = t1[p] * uq + t2[p] * wq + n[p] * zq;
    }
}

// Geometry update (Section 2.3, selective re-assembly of K(u)): the coupling blocks of
// element e for realisation s on its deformed surface X + u_s. The frame (edge vectors,
// normal, in-plane axes, projected coordinates) takes the set-up kernel's binary64
// arithmetic; the blocks take it too for the binary64 form, and binary32 arithmetic on
// the rounded frame for the binary32 forms (coupling_block_f32), which store them in
// binary32. The element matrix is symmetric, so its three off-diagonal corner blocks
// K_01, K_12, K_20 determine the rest (K_ab = K_ba^T); they go to kcs [E][3][9][Sp]
// (sample index innermost). u is read as binary64 from the state of any form. An element
// whose deformed area is zero or not finite sets bit 3 of *flags.
// C / E of the binary32 block arithmetic (C11, C12, C33, C44 as in coupling_block),
// formed once on the host in binary64 and rounded.
struct CoeffsF32 {
    float c11, c12, c33, c44;
};

template <int FORM>
__global__ void reassemble_kernel(const double *__restrict__ xyz, const int32_t *__restrict__ tri,
                                  int32_t E, int32_t Sp, double nu, double ks, const CoeffsF32 cf,
                                  const void *__restrict__ u_main, const void *__restrict__ aux,
                                  void *__restrict__ kcs, int *flags) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)E * Sp) return;
    const int32_t e = (int32_t)(t / Sp);
    const int32_t s = (int32_t)(t - (int64_t)e * Sp);
    double X[3][3];
    for (int j = 0; j < 3; j++) {
        const int64_t node = tri[3 * e + j];
        for (int d = 0; d < 3; d++) {
            const int64_t idx = (node * 3 + d) * Sp + s;
            double u;
            if constexpr (FORM == kKahan32)
                u = f32_to_f64(((const float *)u_main)[idx]) + f32_to_f64(((const float *)aux)[idx]);
            else if constexpr (FORM == kFP32Force)
                u = join_state(((const float *)u_main)[idx], ((const uint32_t *)aux)[idx]);
            else
                u = ((const double *)u_main)[idx];
            X[j][d] = xyz[3 * node + d] + u;
        }
    }
    ElemFrame f;
    if (!element_frame<true>(X, f)) {
        atomicOr(flags, 8);
        return;
    }
    if constexpr (FORM == kFP64) {
        for (int c = 0; c < 3; c++) {  // block c couples corner c to corner (c + 1) mod 3
            double G[3][3];
            coupling_block(f, c, (c + 1) % 3, nu, ks, G);
            for (int r = 0; r < 3; r++)
                for (int q = 0; q < 3; q++)
                    ((double *)kcs)[(((int64_t)e * 3 + c) * 9 + 3 * r + q) * Sp + s] = G[r][q];
        }
    } else {
        const float sc = 0.25f / (float)f.area;
        float t1[3], t2[3], n[3], b[3], g[3];
        for (int d = 0; d < 3; d++) {
            t1[d] = (float)f.t1[d];
            t2[d] = (float)f.t2[d];
            n[d] = (float)f.n[d];
            b[d] = (float)f.b[d];
            g[d] = (float)f.g[d];
        }
        for (int c = 0; c < 3; c++) {  // block c couples corner c to corner (c + 1) mod 3
            const int k = (c + 1) % 3;
            float G[3][3];
            coupling_block_f32(t1, t2, n, b[c], g[c], b[k], g[k], sc, cf.c11, cf.c12, cf.c33, cf.c44, G);
            for (int r = 0; r < 3; r++)
                for (int q = 0; q < 3; q++) ((float *)kcs)[(((int64_t)e * 3 + c) * 9 + 3 * r + q) * Sp + s] = G[r][q];
        }
    }
}

// Three-point Gauss rule (barycentric (2/3, 1/6, 1/6) and permutations, weights 1/3)
// of the product of the linearly interpolated modulus and thickness.
__global__ void setup_eh_kernel(const int32_t *__restrict__ tri, const double *__restrict__ En,
                                const double *__restrict__ hn, int32_t E, int32_t Sp,
                                double *__restrict__ eh) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)E * Sp) return;
    int32_t e = (int32_t)(t / Sp);
    int32_t s = (int32_t)(t - (int64_t)e * Sp);
    double Ev[3], hv[3];
    for (int j = 0; j < 3; j++) {
        int64_t node = tri[3 * e + j];
        Ev[j] = En[node * Sp + s];
        hv[j] = hn[node * Sp + s];
    }
    double acc = 0.0;
    for (int gp = 0; gp < 3; gp++) {
        double Eg = 0.0, hg = 0.0;
        for (int j = 0; j < 3; j++) {
            double lam = (j == gp) ? (2.0 / 3.0) : (1.0 / 6.0);
            Eg += lam * Ev[j];
            hg += lam * hv[j];
        }
        acc += Eg * hg;
    }
    eh[t] = acc / 3.0;
}

// Lumped mass gathered through the node -> element lists: each element gives each of
// its corners rho * A_e * hbar_e / 3 with hbar_e the element-mean thickness.
__global__ void setup_mass_kernel(const int32_t *__restrict__ rowptr, const int4 *__restrict__ ent,
                                  const double *__restrict__ area, const double *__restrict__ hn,
                                  int32_t N, int32_t Sp, double rho, double *__restrict__ m) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * Sp) return;
    int32_t i = (int32_t)(t / Sp);
    int32_t s = (int32_t)(t - (int64_t)i * Sp);
    double hi = hn[(int64_t)i * Sp + s];
    double acc = 0.0;
    for (int32_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
        int4 en = ent[p];
        double hbar = (hi + hn[(int64_t)en.y * Sp + s] + hn[(int64_t)en.z * Sp + s]) / 3.0;
        acc += rho * area[en.x] * hbar / 3.0;
    }
    m[t] = acc;
}

// The same lumped mass from per-element coefficients: each element gives each of its
// corners A_e (rho hbar)_e,s / 3, with (rho hbar)_e,s given by the caller.
__global__ void setup_mass_elem_kernel(const int32_t *__restrict__ rowptr, const int4 *__restrict__ ent,
                                       const double *__restrict__ area, const double *__restrict__ rhoh,
                                       int32_t N, int32_t Sp, double *__restrict__ m) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * Sp) return;
    int32_t i = (int32_t)(t / Sp);
    int32_t s = (int32_t)(t - (int64_t)i * Sp);
    double acc = 0.0;
    for (int32_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
        const int32_t e = ent[p].x;
        acc += area[e] * rhoh[(int64_t)e * Sp + s] / 3.0;
    }
    m[t] = acc;
}

// Element modulus of per-element coefficients for the stress output: E_e,s =
// (E h)_e,s / hbar_e,s with hbar_e,s = (rho hbar)_e,s / rho (E and h constant on the
// element).
__global__ void modulus_from_coeffs_kernel(const double *__restrict__ eh, const double *__restrict__ rhoh,
                                           int64_t n, double rho, double *__restrict__ ebar) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    ebar[t] = eh[t] * rho / rhoh[t];
}

// Per element, over the real samples: omega^2 lower bound (element top eigenvector
// padded with zeros, global lumped masses) and upper bound (element eigenvalue with
// the element's own lumped-mass share, Irons-Treharne).
__global__ void setup_stability_kernel(const int32_t *__restrict__ tri,
                                       const double *__restrict__ eh,
                                       const double *__restrict__ m,
                                       const double *__restrict__ area,
                                       const double *__restrict__ hn,
                                       const double *__restrict__ lam_lo,
                                       const double *__restrict__ lam_hi,
                                       const double *__restrict__ xsq, int32_t E, int32_t S,
                                       int32_t Sp, double rho, const double *__restrict__ rhoh,
                                       double *__restrict__ w2lo, double *__restrict__ w2hi) {
    int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    double lo = 0.0, hi = 0.0;
    if (area[e] > 0.0) {
        for (int32_t s = 0; s < S; s++) {
            double ehs = eh[(int64_t)e * Sp + s];
            double mx = 0.0, hbar = 0.0;
            for (int c = 0; c < 3; c++) {
                int64_t node = tri[3 * e + c];
                mx += m[node * Sp + s] * xsq[3 * e + c];
                if (!rhoh) hbar += hn[node * Sp + s] / 3.0;
            }
            if (mx > 0.0) lo = fmax(lo, ehs * lam_lo[e] / mx);
            // (rhoh: per-element coefficients, the element's own rho hbar)
            double me = rhoh ? area[e] * rhoh[(int64_t)e * Sp + s] / 3.0 : rho * area[e] * hbar / 3.0;
            if (me > 0.0) hi = fmax(hi, ehs * lam_hi[e] / me);
        }
    }
    w2lo[e] = lo;
    w2hi[e] = hi;
}

__global__ void pack_kc_kernel(const double *__restrict__ kc64, int64_t nnz, void *out,
                               int to_float) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nnz * 20) return;
    int64_t p = t / 20;
    int r = (int)(t - p * 20);
    if (to_float) {
        ((float *)out)[t] = r < 18 ? (float)kc64[18 * p + r] : 0.0f;
    } else if (r < 18) {
        ((double *)out)[18 * p + r] = kc64[18 * p + r];
    }
}

__global__ void pack_records_kernel(const float *__restrict__ kc, const int32_t *__restrict__ rowptr,
                                    int32_t N, int32_t nb, int32_t cnt_max, float *__restrict__ kc_rec,
                                    int64_t total) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int64_t per = (int64_t)cnt_max * 20;
    const int64_t b = t / per;
    const int32_t r = (int32_t)(t - b * per);
    const int32_t j = r / 20, q = r - j * 20;
    const int64_t n0 = b * nb;
    const int64_t n1 = n0 + nb < N ? n0 + nb : N;
    const int32_t pb = rowptr[n0];
    const int32_t cnt = rowptr[n1] - pb;
    kc_rec[t] = j < cnt ? kc[((int64_t)pb + j) * 20 + q] : 0.0f;
}

__global__ void convert_kernel(const double *__restrict__ in, int64_t n, void *out, int to_float,
                               int invert) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    double x = invert ? 1.0 / in[t] : in[t];
    if (to_float)
        ((float *)out)[t] = (float)x;
    else
        ((double *)out)[t] = x;
}

// dst [N][Sp] = src [N][S], padding samples repeating sample 0; counts entries of src
// that are not finite and > 0 into *bad.
__global__ void pad_fields_kernel(const double *__restrict__ src, int32_t N, int32_t S, int32_t Sp,
                                  double *__restrict__ dst, int *bad) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * Sp) return;
    const int64_t i = t / Sp;
    const int32_t s = (int32_t)(t - i * Sp);
    const double x = src[i * S + (s < S ? s : 0)];
    if (s < S && !(isfinite(x) && x > 0.0)) atomicAdd(bad, 1);
    dst[t] = x;
}

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t launch_setup_elements(const double *xyz, const int32_t *tri, const int32_t *ec2ent,
                                  int32_t E, double nu, double kshear, double *kc64,
                                  double *area, double *lam_lo, double *lam_hi, double *xsq,
                                  double *kfull, int *bad, cudaStream_t s) {
    if (E == 0) return cudaSuccess;
    setup_elements_kernel<<<blocks_for(E, 128), 128, 0, s>>>(xyz, tri, ec2ent, E, nu, kshear,
                                                              kc64, area, lam_lo, lam_hi, xsq,
                                                              kfull, bad);
    return cudaGetLastError();
}

cudaError_t launch_reassemble(int form, const double *xyz, const int32_t *tri, int32_t E, int32_t Sp, double nu,
                              double kshear, const void *u_main, const void *aux, void *kcs, int *flags,
                              cudaStream_t s) {
    const int64_t n = (int64_t)E * Sp;
    if (n == 0) return cudaSuccess;
    const unsigned g = blocks_for(n, 128);
    const double C11 = 1.0 / (1.0 - nu * nu);
    const CoeffsF32 cf{(float)C11, (float)(nu * C11), (float)(0.5 * (1.0 - nu) * C11),
                       (float)(0.5 * kshear * (1.0 - nu) * C11)};
    if (form == kFP64)
        reassemble_kernel<kFP64><<<g, 128, 0, s>>>(xyz, tri, E, Sp, nu, kshear, cf, u_main, aux, kcs, flags);
    else if (form == kFP32Force)
        reassemble_kernel<kFP32Force><<<g, 128, 0, s>>>(xyz, tri, E, Sp, nu, kshear, cf, u_main, aux, kcs, flags);
    else
        reassemble_kernel<kKahan32><<<g, 128, 0, s>>>(xyz, tri, E, Sp, nu, kshear, cf, u_main, aux, kcs, flags);
    return cudaGetLastError();
}

cudaError_t launch_setup_eh(const int32_t *tri, const double *E_node, const double *h_node,
                            int32_t E, int32_t Sp, double *eh64, cudaStream_t s) {
    int64_t n = (int64_t)E * Sp;
    if (n == 0) return cudaSuccess;
    setup_eh_kernel<<<blocks_for(n, 256), 256, 0, s>>>(tri, E_node, h_node, E, Sp, eh64);
    return cudaGetLastError();
}

cudaError_t launch_setup_mass(const int32_t *rowptr, const int4 *ent, const double *area,
                              const double *h_node, int32_t N, int32_t Sp, double rho,
                              double *m64, cudaStream_t s) {
    int64_t n = (int64_t)N * Sp;
    if (n == 0) return cudaSuccess;
    setup_mass_kernel<<<blocks_for(n, 256), 256, 0, s>>>(rowptr, ent, area, h_node, N, Sp, rho,
                                                         m64);
    return cudaGetLastError();
}

cudaError_t launch_setup_stability(const int32_t *tri, const double *eh64, const double *m64,
                                   const double *area, const double *h_node,
                                   const double *lam_lo, const double *lam_hi,
                                   const double *xsq, int32_t E, int32_t S, int32_t Sp,
                                   double rho, const double *rhoh, double *w2lo, double *w2hi,
                                   cudaStream_t s) {
    if (E == 0) return cudaSuccess;
    setup_stability_kernel<<<blocks_for(E, 128), 128, 0, s>>>(tri, eh64, m64, area, h_node,
                                                               lam_lo, lam_hi, xsq, E, S, Sp,
                                                               rho, rhoh, w2lo, w2hi);
    return cudaGetLastError();
}

cudaError_t launch_setup_mass_elem(const int32_t *rowptr, const int4 *ent, const double *area,
                                   const double *rhoh, int32_t N, int32_t Sp, double *m64, cudaStream_t s) {
    int64_t n = (int64_t)N * Sp;
    if (n == 0) return cudaSuccess;
    setup_mass_elem_kernel<<<blocks_for(n, 256), 256, 0, s>>>(rowptr, ent, area, rhoh, N, Sp, m64);
    return cudaGetLastError();
}

cudaError_t launch_modulus_from_coeffs(const double *eh64, const double *rhoh, int64_t n, double rho,
                                       double *ebar, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    modulus_from_coeffs_kernel<<<blocks_for(n, 256), 256, 0, s>>>(eh64, rhoh, n, rho, ebar);
    return cudaGetLastError();
}

cudaError_t launch_pack_kc(const double *kc64, int64_t nnz, void *kc_out, int to_float,
                           cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    pack_kc_kernel<<<blocks_for(nnz * 20, 256), 256, 0, s>>>(kc64, nnz, kc_out, to_float);
    return cudaGetLastError();
}

cudaError_t launch_pack_records(const float *kc, const int32_t *rowptr, int32_t N, int32_t nb,
                                int32_t cnt_max, float *kc_rec, cudaStream_t s) {
    const int64_t total = (int64_t)((N + nb - 1) / nb) * cnt_max * 20;
    if (total == 0) return cudaSuccess;
    pack_records_kernel<<<blocks_for(total, 256), 256, 0, s>>>(kc, rowptr, N, nb, cnt_max, kc_rec, total);
    return cudaGetLastError();
}

cudaError_t launch_pad_fields(const double *src, int32_t N, int32_t S, int32_t Sp, double *dst,
                              int *bad, cudaStream_t s) {
    const int64_t n = (int64_t)N * Sp;
    if (n == 0) return cudaSuccess;
    pad_fields_kernel<<<blocks_for(n, 256), 256, 0, s>>>(src, N, S, Sp, dst, bad);
    return cudaGetLastError();
}

cudaError_t launch_convert(const double *in, int64_t n, void *out, int to_float, int invert,
                           cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    convert_kernel<<<blocks_for(n, 256), 256, 0, s>>>(in, n, out, to_float, invert);
    return cudaGetLastError();
}

}  // namespace ens
