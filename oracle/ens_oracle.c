/*
 * FP64 CPU oracle for the explicit ensemble update of the segregated wall model
 * (Li & Schiavazzi, "An ensemble solver for segregated cardiovascular FSI").
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct reference
 * that the CUDA library is checked against. Only the test suite, the smoke check and
 * the benchmark's CPU-baseline arm may load it; the library never does, and this file
 * shares no source with the library.
 *
 * Layout: every per-sample array is sample-OUTERMOST, e.g. u[s][node][dof], so that each
 * realisation reads like an independent deterministic solve.
 *
 * What each function follows:
 *   orc_element_matrices : Section 2.2.1, the strain-displacement matrix B (Eq. eps = B u),
 *                          the constitutive matrix C, and k_e = sum_gp B^T C B A_e zeta w.
 *   orc_gauss_eh         : Section 2.2.1, three-point Gauss rule with E and zeta varying
 *                          linearly inside each element.
 *   orc_lumped_mass      : Section 2.3, lumped mass matrix M~ pre-assembled before the loop.
 *   orc_internal_force   : K u as the sum of element products (assembly free, Section 2.4).
 *   orc_cd_start/steps   : Section 2.3, central-difference update Eq. (dynamicsCD), with
 *                          C = alpha M.
 *   orc_stats            : ensemble mean and sample variance (Section 3.1 reports ensemble
 *                          means and confidence bands), plain two-pass formula.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/*
 * One element: global-frame stiffness per unit (E * thickness), 9 x 9, dof order
 * (ux1, uy1, uz1, ux2, ..., uz3).
 *
 * Local frame (the paper names a local shell frame but does not define it): e1 along
 * edge 1->2, n the unit normal (X2-X1) x (X3-X1), e2 = n x e1. Local coordinates of the
 * corners are x_j = (X_j - X1).e1, y_j = (X_j - X1).e2.
 *
 * B is the 5 x 9 matrix of Section 2.2.1 (rows eps_xx, eps_yy, gamma_xy, gamma_xz,
 * gamma_yz) with x_ij = x_i - x_j, scaled by 1 / (2 A_e). C0 = C / E is the constitutive
 * matrix of Section 2.2.1 without E. With E and zeta linear in the element and the Gauss
 * weights normalised to sum to one, k_e = A_e B^T C0 B * (E zeta)_e where
 * (E zeta)_e = sum_gp w_gp E(gp) zeta(gp) (orc_gauss_eh). The local matrix is rotated to
 * the global frame as T^T K_local T with T = blockdiag(L, L, L), L rows = (e1, e2, n).
 *
 * Returns 0, or -1 for a degenerate triangle.
 */
int orc_element_matrix(const double *X, double nu, double kshear, double *Kg, double *area_out)
{
    double a[3], b[3], n[3], e1[3], e2[3];
    for (int d = 0; d < 3; d++) {
        a[d] = X[3 + d] - X[d];
        b[d] = X[6 + d] - X[d];
    }
    cross3(a, b, n);
    double nn = sqrt(dot3(n, n));
    double la = sqrt(dot3(a, a));
    if (!(nn > 0.0) || !(la > 0.0))
        return -1;
    double A = 0.5 * nn;
    for (int d = 0; d < 3; d++) {
        n[d] /= nn;
        e1[d] = a[d] / la;
    }
    cross3(n, e1, e2);

    double x[3], y[3];
    for (int j = 0; j < 3; j++) {
        double r[3] = {X[3 * j] - X[0], X[3 * j + 1] - X[1], X[3 * j + 2] - X[2]};
        x[j] = dot3(r, e1);
        y[j] = dot3(r, e2);
    }
    double y23 = y[1] - y[2], y31 = y[2] - y[0], y12 = y[0] - y[1];
    double x32 = x[2] - x[1], x13 = x[0] - x[2], x21 = x[1] - x[0];

    double B[5][9];
    memset(B, 0, sizeof(B));
    double byx[3] = {y23, y31, y12}; /* d/dx of the shape functions times 2A */
    double bxy[3] = {x32, x13, x21}; /* d/dy of the shape functions times 2A */
    for (int j = 0; j < 3; j++) {
        B[0][3 * j + 0] = byx[j];
        B[1][3 * j + 1] = bxy[j];
        B[2][3 * j + 0] = bxy[j];
        B[2][3 * j + 1] = byx[j];
        B[3][3 * j + 2] = byx[j];
        B[4][3 * j + 2] = bxy[j];
    }
    for (int r = 0; r < 5; r++)
        for (int c = 0; c < 9; c++)
            B[r][c] /= (2.0 * A);

    double C0[5][5];
    memset(C0, 0, sizeof(C0));
    double f = 1.0 / (1.0 - nu * nu);
    C0[0][0] = f;
    C0[0][1] = f * nu;
    C0[1][0] = f * nu;
    C0[1][1] = f;
    C0[2][2] = f * 0.5 * (1.0 - nu);
    C0[3][3] = f * 0.5 * kshear * (1.0 - nu);
    C0[4][4] = f * 0.5 * kshear * (1.0 - nu);

    /* K_local = A * B^T C0 B */
    double CB[5][9];
    for (int r = 0; r < 5; r++)
        for (int c = 0; c < 9; c++) {
            double s = 0.0;
            for (int k = 0; k < 5; k++)
                s += C0[r][k] * B[k][c];
            CB[r][c] = s;
        }
    double Kl[9][9];
    for (int i = 0; i < 9; i++)
        for (int j = 0; j < 9; j++) {
            double s = 0.0;
            for (int k = 0; k < 5; k++)
                s += B[k][i] * CB[k][j];
            Kl[i][j] = A * s;
        }

    /* T = blockdiag(L, L, L), u_local = T u_global, K_global = T^T K_local T */
    double L[3][3];
    for (int d = 0; d < 3; d++) {
        L[0][d] = e1[d];
        L[1][d] = e2[d];
        L[2][d] = n[d];
    }
    double T[9][9];
    memset(T, 0, sizeof(T));
    for (int blk = 0; blk < 3; blk++)
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++)
                T[3 * blk + r][3 * blk + c] = L[r][c];
    double KT[9][9];
    for (int i = 0; i < 9; i++)
        for (int j = 0; j < 9; j++) {
            double s = 0.0;
            for (int k = 0; k < 9; k++)
                s += Kl[i][k] * T[k][j];
            KT[i][j] = s;
        }
    for (int i = 0; i < 9; i++)
        for (int j = 0; j < 9; j++) {
            double s = 0.0;
            for (int k = 0; k < 9; k++)
                s += T[k][i] * KT[k][j];
            Kg[9 * i + j] = s;
        }
    if (area_out)
        *area_out = A;
    return 0;
}

/* All elements: Kg [E][81], area [E]. Returns 0, or -(1 + e) for the first degenerate e. */
int orc_element_matrices(int32_t n_elems, const double *xyz, const int32_t *tri, double nu,
                         double kshear, double *Kg, double *area)
{
    int bad = -1;
#pragma omp parallel for schedule(static)
    for (int32_t e = 0; e < n_elems; e++) {
        double X[9];
        for (int j = 0; j < 3; j++)
            for (int d = 0; d < 3; d++)
                X[3 * j + d] = xyz[3 * (int64_t)tri[3 * e + j] + d];
        if (orc_element_matrix(X, nu, kshear, Kg + 81 * (int64_t)e, area + e) != 0) {
#pragma omp critical
            if (bad < 0 || e < bad)
                bad = e;
        }
    }
    return bad < 0 ? 0 : -(1 + bad);
}

/*
 * Gauss-point products. Three-point rule with the points at barycentric (2/3, 1/6, 1/6)
 * and its permutations, weights 1/3 each (normalised: the element area enters k_e
 * separately). E and zeta are interpolated linearly from the nodal values.
 *   eh[s][e]   = sum_gp w E(gp) zeta(gp)
 *   hbar[s][e] = sum_gp w zeta(gp)
 * E_node, h_node: [S][N].
 */
void orc_gauss_eh(int32_t n_nodes, int32_t n_elems, int32_t S, const int32_t *tri,
                  const double *E_node, const double *h_node, double *eh, double *hbar)
{
    static const double lam[3][3] = {
        {2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0},
        {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0},
        {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0},
    };
#pragma omp parallel for collapse(2) schedule(static)
    for (int32_t s = 0; s < S; s++)
        for (int32_t e = 0; e < n_elems; e++) {
            const double *Es = E_node + (int64_t)s * n_nodes;
            const double *hs = h_node + (int64_t)s * n_nodes;
            double acc = 0.0, acch = 0.0;
            for (int g = 0; g < 3; g++) {
                double Eg = 0.0, hg = 0.0;
                for (int j = 0; j < 3; j++) {
                    Eg += lam[g][j] * Es[tri[3 * e + j]];
                    hg += lam[g][j] * hs[tri[3 * e + j]];
                }
                acc += (1.0 / 3.0) * Eg * hg;
                acch += (1.0 / 3.0) * hg;
            }
            eh[(int64_t)s * n_elems + e] = acc;
            hbar[(int64_t)s * n_elems + e] = acch;
        }
}

/* Lumped mass per node and sample: m[s][i] = sum over elements e touching i of rho A_e hbar[s][e] / 3. */
void orc_lumped_mass(int32_t n_nodes, int32_t n_elems, int32_t S, const int32_t *tri,
                     const double *area, const double *hbar, double rho, double *m)
{
#pragma omp parallel for schedule(static)
    for (int32_t s = 0; s < S; s++) {
        double *ms = m + (int64_t)s * n_nodes;
        for (int32_t i = 0; i < n_nodes; i++)
            ms[i] = 0.0;
        for (int32_t e = 0; e < n_elems; e++) {
            double me = rho * area[e] * hbar[(int64_t)s * n_elems + e] / 3.0;
            for (int j = 0; j < 3; j++)
                ms[tri[3 * e + j]] += me;
        }
    }
}

/* One sample's internal force f = K_s u = sum_e (E zeta)_e,s Kg_e u_e, scattered to nodes. */
static void internal_force_one(int32_t n_nodes, int32_t n_elems, const int32_t *tri, const double *Kg,
                               const double *eh_s, const double *u, double *f)
{
    memset(f, 0, sizeof(double) * 3 * (size_t)n_nodes);
    for (int32_t e = 0; e < n_elems; e++) {
        double ue[9], fe[9];
        for (int j = 0; j < 3; j++)
            for (int d = 0; d < 3; d++)
                ue[3 * j + d] = u[3 * (int64_t)tri[3 * e + j] + d];
        const double *K = Kg + 81 * (int64_t)e;
        for (int r = 0; r < 9; r++) {
            double s = 0.0;
            for (int c = 0; c < 9; c++)
                s += K[9 * r + c] * ue[c];
            fe[r] = eh_s[e] * s;
        }
        for (int j = 0; j < 3; j++)
            for (int d = 0; d < 3; d++)
                f[3 * (int64_t)tri[3 * e + j] + d] += fe[3 * j + d];
    }
}

/* f[s][i][d] = (K_s u_s)[i][d] for all samples; u, f: [S][N][3]. */
void orc_internal_force(int32_t n_nodes, int32_t n_elems, int32_t S, const int32_t *tri,
                        const double *Kg, const double *eh, const double *u, double *f)
{
#pragma omp parallel for schedule(static)
    for (int32_t s = 0; s < S; s++)
        internal_force_one(n_nodes, n_elems, tri, Kg, eh + (int64_t)s * n_elems,
                           u + (int64_t)s * 3 * n_nodes, f + (int64_t)s * 3 * n_nodes);
}

/* External nodal force at one step: f[i][d] = sum_j amp_row[j] modes[j][i][d]. */
static void external_force(int32_t n_nodes, int32_t J, const double *modes, const double *amp_row,
                           double *f)
{
    for (int64_t k = 0; k < 3 * (int64_t)n_nodes; k++) {
        double s = 0.0;
        for (int32_t j = 0; j < J; j++)
            s += amp_row[j] * modes[(int64_t)j * 3 * n_nodes + k];
        f[k] = s;
    }
}

/*
 * Start of the central-difference recursion. The paper does not state how u_{-1} is
 * obtained; the oracle takes the textbook Taylor start
 *   u_{-1} = u_0 - dt v_0 + (dt^2 / 2) a_0,  a_0 = M^-1 (f_0 - K u_0 - C v_0),  C = alpha M.
 * Fixed dofs are held at zero (u_{-1} = 0 there).
 */
void orc_cd_start(int32_t n_nodes, int32_t n_elems, int32_t S, const int32_t *tri, const double *Kg,
                  const double *eh, const double *m, double alpha, double dt, const uint8_t *fixed,
                  int32_t J, const double *modes, const double *amp0, const double *u0,
                  const double *v0, double *u_prev)
{
    double *fext = (double *)malloc(sizeof(double) * 3 * (size_t)n_nodes);
    external_force(n_nodes, J, modes, amp0, fext);
#pragma omp parallel for schedule(static)
    for (int32_t s = 0; s < S; s++) {
        const double *us = u0 + (int64_t)s * 3 * n_nodes;
        const double *vs = v0 + (int64_t)s * 3 * n_nodes;
        const double *ms = m + (int64_t)s * n_nodes;
        double *fint = (double *)malloc(sizeof(double) * 3 * (size_t)n_nodes);
        internal_force_one(n_nodes, n_elems, tri, Kg, eh + (int64_t)s * n_elems, us, fint);
        for (int32_t i = 0; i < n_nodes; i++)
            for (int d = 0; d < 3; d++) {
                int64_t k = 3 * (int64_t)i + d;
                double a0 = (fext[k] - fint[k] - alpha * ms[i] * vs[k]) / ms[i];
                double up = us[k] - dt * vs[k] + 0.5 * dt * dt * a0;
                u_prev[(int64_t)s * 3 * n_nodes + k] = fixed[k] ? 0.0 : up;
            }
        free(fint);
    }
    free(fext);
}

/*
 * n_steps steps of Eq. (dynamicsCD) with lumped M and C = alpha M:
 *   (M + dt/2 C) u_{n+1} = dt^2 f_n - (dt^2 K - 2 M) u_n - (M - dt/2 C) u_{n-1}
 * starting at step index step0 (the load row used for step n is amp[n]). On entry
 * u_prev = u_{step0 - 1}, u_cur = u_{step0}; on return they hold the last two states.
 * Fixed dofs are held at zero. Returns 0, or -1 if the amplitude table is too short.
 */
int orc_cd_steps(int32_t n_nodes, int32_t n_elems, int32_t S, const int32_t *tri, const double *Kg,
                 const double *eh, const double *m, double alpha, double dt, const uint8_t *fixed,
                 int32_t J, const double *modes, int64_t n_amp, const double *amp, int64_t step0,
                 int64_t n_steps, double *u_prev, double *u_cur)
{
    if (step0 < 0 || step0 + n_steps > n_amp)
        return -1;
    int64_t n3 = 3 * (int64_t)n_nodes;
    double *fext = (double *)malloc(sizeof(double) * n3);
#pragma omp parallel
    {
        double *fint = (double *)malloc(sizeof(double) * n3);
        double *unext = (double *)malloc(sizeof(double) * n3);
        for (int64_t n = step0; n < step0 + n_steps; n++) {
#pragma omp single
            external_force(n_nodes, J, modes, amp + n * J, fext);
#pragma omp for schedule(static)
            for (int32_t s = 0; s < S; s++) {
                double *up = u_prev + (int64_t)s * n3;
                double *uc = u_cur + (int64_t)s * n3;
                const double *ms = m + (int64_t)s * n_nodes;
                internal_force_one(n_nodes, n_elems, tri, Kg, eh + (int64_t)s * n_elems, uc, fint);
                for (int32_t i = 0; i < n_nodes; i++) {
                    double M = ms[i], C = alpha * ms[i];
                    for (int d = 0; d < 3; d++) {
                        int64_t k = 3 * (int64_t)i + d;
                        double rhs = dt * dt * fext[k] - (dt * dt * fint[k] - 2.0 * M * uc[k])
                                     - (M - 0.5 * dt * C) * up[k];
                        unext[k] = fixed[k] ? 0.0 : rhs / (M + 0.5 * dt * C);
                    }
                }
                memcpy(up, uc, sizeof(double) * n3);
                memcpy(uc, unext, sizeof(double) * n3);
            }
        }
        free(fint);
        free(unext);
    }
    free(fext);
    return 0;
}

/* Ensemble mean and sample variance (divisor S - 1; 0 when S == 1) of u[s][k], two passes. */
void orc_stats(int32_t S, int64_t n, const double *u, double *mean, double *var)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; k++) {
        double s = 0.0;
        for (int32_t j = 0; j < S; j++)
            s += u[(int64_t)j * n + k];
        double mu = S > 0 ? s / S : 0.0;
        double q = 0.0;
        for (int32_t j = 0; j < S; j++) {
            double d = u[(int64_t)j * n + k] - mu;
            q += d * d;
        }
        mean[k] = mu;
        var[k] = S > 1 ? q / (S - 1) : 0.0;
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
