/*
 * oracle.h -- plain FP64 CPU oracle for the single-projection PCA motion solve
 * of Li et al., "3D tumor localization through real-time volumetric x-ray
 * imaging for lung cancer radiotherapy" (arXiv:1102.1712).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The CUDA product
 * path never links, calls or includes anything from here, and nothing here is
 * shared with it (geometry, sampling rule, interpolation and reductions are
 * each written out again, independently, on both sides).
 *
 * Every routine works on host memory in double precision and follows the
 * paper's definitions step by step, with no blocking, fusion or reordering:
 *   Eq. (1)         DVF synthesis x = xbar + U w
 *   Eq. (A.3/A.5)   trilinear warp f(v) = f0(v + x(v))
 *   Eq. (2)         cost ||P f - a y - b||^2 with projector P
 *   Eq. (A.1)       intensity scaling (a, b) by least squares on Y = [y, 1]
 *   Eq. (A.2), Appendix  normalised gradient step with Armijo backtracking
 *   gradient below Eq. (A.2)  dJ/dw = 2 U^T (df/dx) P^T (P f - a y - b)
 *   Eq. (A.8)       warp Jacobian (right derivative at grid lines)
 *   Eq. (3)         linear prediction of w from the last L solutions
 *   Sec. II.A       tumour localisation by fixed-point DVF inversion
 *
 * Readings where the paper is silent (all pinned by tests, see the test
 * files): 0-based indices, DVF stored in mm and divided by the voxel spacing,
 * zero outside the grid; a source-anchored trilinear ray march as P (samples
 * t_i = i*step along the unit ray, kept while inside the support box
 * [-1, n] in voxel units); gantry about z through the world origin.
 *
 * Return codes match the product library: 0 ok, 1 invalid argument,
 * 2 singular Y^T Y, 4 not converged (informational).
 */
#ifndef PCAS_ORACLE_H
#define PCAS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Volume: voxel (i,j,k) centre at (ox + i*sx, oy + j*sy, oz + k*sz) mm,
 * data index (k*ny + j)*nx + i. */
typedef struct { int nx, ny, nz; double sx, sy, sz, ox, oy, oz; } ovol;

/* Cone-beam view.  Source S = (sad sin a, -sad cos a, 0); the detector
 * plane is normal to the central ray at distance sdd from S; pixel (iu, iv)
 * centre = S + sdd*ew + ((iu-(nu-1)/2)du + off_u) eu + ((iv-(nv-1)/2)dv + off_v) ev
 * with ew = (-sin a, cos a, 0), eu = (cos a, sin a, 0), ev = (0, 0, 1).
 * Image layout [nv][nu], u fastest. */
typedef struct { double sad, sdd; int nu, nv; double du, dv, off_u, off_v, angle; } ocb;

/* Solver constants (Appendix, after Eq. A.2). */
typedef struct { double mu0, alpha, beta, mu_min; int max_iter, max_trials; double step; } oparams;

typedef struct { int iters, evals, status; double J0, J, a, b, mu_last; } ostats;

/* Eq. (1). dvf is [3][N] mm. mean may be NULL (zero mean). */
int oracle_pca_dvf(const double* mean, const double* U, int K, const double* w,
                   const ovol* vol, double* dvf);
/* Eq. (A.3)/(A.5): f(v) = f0(v + x(v)/s), zero outside the grid. */
int oracle_warp_volume(const double* f0, const double* dvf, const ovol* vol, double* f);
/* Eq. (A.5) at one continuous voxel-unit point (exposed for tests). */
double oracle_trilinear(const double* f, const ovol* vol, double q1, double q2, double q3);
/* Eq. (A.8) and its y/z analogues at one point: dfdq[c] = d f / d q_c. */
void oracle_trilinear_grad(const double* f, const ovol* vol, double q1, double q2,
                           double q3, double dfdq[3]);
/* P: p[iv*nu+iu] = step * sum_i f(S + i*step*dhat), over samples in the support box. */
int oracle_drr_forward(const double* f, const ovol* vol, const ocb* cb, double step, double* p);
/* One ray of P (sampled parity checks at full size). */
double oracle_drr_ray(const double* f, const ovol* vol, const ocb* cb, double step, int iu, int iv);
/* Siddon's exact radiological path (Sec. II.B renders its simulated projections
 * with it): the integral of the piecewise-constant volume (voxel (i,j,k) = its
 * value on the cube of side s centred on it, zero outside) along the ray from
 * S through the centre of pixel (iu, iv).  Plane crossings of the ray with all
 * voxel faces, sorted; each segment between consecutive crossings adds its
 * length times the value of the voxel containing its midpoint. */
int oracle_siddon_forward(const double* f, const ovol* vol, const ocb* cb, double* p);
double oracle_siddon_ray(const double* f, const ovol* vol, const ocb* cb, int iu, int iv);
/* P^T: the literal transpose of oracle_drr_forward (scatter form). g overwritten. */
int oracle_drr_adjoint(const double* img, const ovol* vol, const ocb* cb, double step, double* g);
/* Eq. (A.1): least squares of p on [y, 1]. Returns 2 if Y^T Y is singular. */
int oracle_intensity_fit(const double* p, const double* y, long M, double* a, double* b);
/* Eq. (2) for given (a, b). */
double oracle_cost(const double* p, const double* y, long M, double a, double b);
/* Cost and gradient at w.  If fit_ab != 0, (a, b) come from Eq. (A.1) at w
 * and are returned in ab; otherwise ab[0], ab[1] are used as given. */
int oracle_cost_grad(const double* f0, const double* mean, const double* U, int K,
                     const double* w, const double* y, const ovol* vol, const ocb* cb,
                     double step, int fit_ab, double* ab, double* J, double* G);
/* Forward-mode form of the same gradient: G_k = 2 <r, P h_k> with
 * h_k(v) = sum_c (df/dq_c)(v) u_kc(v) / s_c.  Exposed as an independent check. */
int oracle_grad_forward_mode(const double* f0, const double* mean, const double* U, int K,
                             const double* w, const double* y, const ovol* vol,
                             const ocb* cb, double step, double a, double b, double* G);
/* Transpose of the warp of Eq. (A.5) for a fixed DVF: out[u] = sum_v z[v] *
 * (trilinear weight of tap u at q(v)), i.e. <W x, z> = <x, W^T z>.  out
 * overwritten (N doubles). */
int oracle_warp_adjoint(const double* z, const double* dvf, const ovol* vol, double* out);
/* Gradient of Eq. (2) with respect to the reference CT at fixed w and (a, b):
 * dJ/df0 = W^T (2 P^T r), r = P W f0 - a y - b.  (a, b) from Eq. (A.1) at w
 * when fit_ab != 0 (returned in ab).  Also returns J. */
int oracle_cost_grad_f0(const double* f0, const double* mean, const double* U, int K,
                        const double* w, const double* y, const ovol* vol, const ocb* cb,
                        double step, int fit_ab, double* ab, double* J, double* dJdf0);
/* Appendix: alternate (A.1) and (A.2) with Armijo backtracking.
 * J_trace (may be NULL) receives the cost after each iteration (max_iter+1). */
int oracle_solve_projection(const double* f0, const double* mean, const double* U, int K,
                            const double* y, const ovol* vol, const ocb* cb,
                            const double* w_init, const oparams* prm, double* w_out,
                            ostats* st, double* J_trace);
/* The same solve, also recording each iteration that reaches the line search
 * (||G|| > 0; row it of it_log, ORACLE_LOG_STRIDE(K) doubles; rows not reached are left
 * as the caller set them): J, a, b at the iterate (after Eq. A.1), ||G||, the
 * accepted step size (0 if none), the trials tried in the iteration, 1 if a
 * step was accepted (else 0), then the iterate w (K), G (K) and d (K). */
#define ORACLE_LOG_STRIDE(K) (7 + 3 * (K))
int oracle_solve_projection_log(const double* f0, const double* mean, const double* U, int K,
                                const double* y, const ovol* vol, const ocb* cb,
                                const double* w_init, const oparams* prm, double* w_out,
                                ostats* st, double* J_trace, double* it_log);
/* Sec. II.A: solve c + x(c) = c_ref by y <- -x(c_ref + y). */
int oracle_localize_tumor(const double* mean, const double* U, int K, const double* w,
                          const ovol* vol, const double c_ref[3], int max_iter,
                          double tol_mm, double c_out[3]);
/* Eq. (3): per-coefficient least-squares fit of c[k*L + (l-1)]. trace is T x K. */
int oracle_lp_fit(const double* trace, int T, int K, int L, double* c);
/* Eq. (3): w0_k = sum_l c_kl hist[(l-1)*K + k]. */
int oracle_lp_predict(const double* hist, const double* c, int K, int L, double* w0);

#ifdef __cplusplus
}
#endif
#endif
