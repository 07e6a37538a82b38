/*
 * oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * Slow and literal on purpose: each function is the paper's definition
 * written out, so it can be checked against the text by eye.  It shares no
 * code with the CUDA path.  OpenMP splits only loops whose iterations share no
 * sum (rays of the forward projectors, voxels of the DVF, the warp and the
 * forward-mode Jacobian), so no result depends on the thread count; the P^T
 * scatter and every reduction run serially in their written order.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static long nvox(const ovol* v) { return (long)v->nx * v->ny * v->nz; }

static int vol_ok(const ovol* v) {
    return v && v->nx > 0 && v->ny > 0 && v->nz > 0 && v->sx > 0 && v->sy > 0 && v->sz > 0;
}

/* ------------------------------------------------------------------ Eq. (1) */
int oracle_pca_dvf(const double* mean, const double* U, int K, const double* w,
                   const ovol* vol, double* dvf) {
    if (!vol_ok(vol) || K < 0 || (K > 0 && (!U || !w)) || !dvf) return 1;
    long N = nvox(vol);
    /* independent voxels: the threads share no sum */
    for (int c = 0; c < 3; c++) {
#pragma omp parallel for schedule(static)
        for (long n = 0; n < N; n++) {
            double x = mean ? mean[c * N + n] : 0.0;
            for (int k = 0; k < K; k++) x += U[((long)k * 3 + c) * N + n] * w[k];
            dvf[c * N + n] = x;
        }
    }
    return 0;
}

/* Voxel value with zero outside the grid (reading of "within the bounding box",
 * Appendix before Eq. A.3). */
static double voxel(const double* f, const ovol* v, long i, long j, long k) {
    if (i < 0 || j < 0 || k < 0 || i >= v->nx || j >= v->ny || k >= v->nz) return 0.0;
    return f[(k * v->ny + j) * v->nx + i];
}

/* ---------------------------------------------------------------- Eq. (A.5) */
double oracle_trilinear(const double* f0, const ovol* vol, double q1, double q2, double q3) {
    double fl = floor(q1), fm = floor(q2), fn = floor(q3);
    long l = (long)fl, m = (long)fm, n = (long)fn;
    double z1 = q1 - fl, z2 = q2 - fm, z3 = q3 - fn;
    return voxel(f0, vol, l, m, n) * (1 - z1) * (1 - z2) * (1 - z3)
         + voxel(f0, vol, l + 1, m, n) * z1 * (1 - z2) * (1 - z3)
         + voxel(f0, vol, l, m + 1, n) * (1 - z1) * z2 * (1 - z3)
         + voxel(f0, vol, l, m, n + 1) * (1 - z1) * (1 - z2) * z3
         + voxel(f0, vol, l + 1, m + 1, n) * z1 * z2 * (1 - z3)
         + voxel(f0, vol, l + 1, m, n + 1) * z1 * (1 - z2) * z3
         + voxel(f0, vol, l, m + 1, n + 1) * (1 - z1) * z2 * z3
         + voxel(f0, vol, l + 1, m + 1, n + 1) * z1 * z2 * z3;
}

/* ---------------------------------------------------------------- Eq. (A.8)
 * d f / d q_1 as printed, and the analogous y and z expressions.  The floor
 * convention makes this the right derivative on grid lines. */
void oracle_trilinear_grad(const double* f0, const ovol* vol, double q1, double q2,
                           double q3, double d[3]) {
    double fl = floor(q1), fm = floor(q2), fn = floor(q3);
    long l = (long)fl, m = (long)fm, n = (long)fn;
    double z1 = q1 - fl, z2 = q2 - fm, z3 = q3 - fn;
#define F0(a, b, c) voxel(f0, vol, (a), (b), (c))
    d[0] = (F0(l + 1, m, n) - F0(l, m, n)) * (1 - z2) * (1 - z3)
         + (F0(l + 1, m + 1, n) - F0(l, m + 1, n)) * z2 * (1 - z3)
         + (F0(l + 1, m, n + 1) - F0(l, m, n + 1)) * (1 - z2) * z3
         + (F0(l + 1, m + 1, n + 1) - F0(l, m + 1, n + 1)) * z2 * z3;
    d[1] = (F0(l, m + 1, n) - F0(l, m, n)) * (1 - z1) * (1 - z3)
         + (F0(l + 1, m + 1, n) - F0(l + 1, m, n)) * z1 * (1 - z3)
         + (F0(l, m + 1, n + 1) - F0(l, m, n + 1)) * (1 - z1) * z3
         + (F0(l + 1, m + 1, n + 1) - F0(l + 1, m, n + 1)) * z1 * z3;
    d[2] = (F0(l, m, n + 1) - F0(l, m, n)) * (1 - z1) * (1 - z2)
         + (F0(l + 1, m, n + 1) - F0(l + 1, m, n)) * z1 * (1 - z2)
         + (F0(l, m + 1, n + 1) - F0(l, m + 1, n)) * (1 - z1) * z2
         + (F0(l + 1, m + 1, n + 1) - F0(l + 1, m + 1, n)) * z1 * z2;
#undef F0
}

/* ------------------------------------------------------ Eq. (A.3) with mm DVF */
int oracle_warp_volume(const double* f0, const double* dvf, const ovol* vol, double* f) {
    if (!vol_ok(vol) || !f0 || !dvf || !f) return 1;
    long N = nvox(vol);
    /* independent voxels: the threads share no sum */
#pragma omp parallel for schedule(static)
    for (long k = 0; k < vol->nz; k++)
        for (long j = 0; j < vol->ny; j++)
            for (long i = 0; i < vol->nx; i++) {
                long n = (k * vol->ny + j) * vol->nx + i;
                double q1 = i + dvf[0 * N + n] / vol->sx;
                double q2 = j + dvf[1 * N + n] / vol->sy;
                double q3 = k + dvf[2 * N + n] / vol->sz;
                f[n] = oracle_trilinear(f0, vol, q1, q2, q3);
            }
    return 0;
}

/* ------------------------------------------------------------- geometry
 * Cone-beam view about the z axis through the world origin. */
typedef struct { double S[3], ew[3], eu[3], ev[3]; } oframe;

static void view_frame(const ocb* cb, oframe* F) {
    double s = sin(cb->angle), c = cos(cb->angle);
    F->S[0] = cb->sad * s;  F->S[1] = -cb->sad * c; F->S[2] = 0.0;
    F->ew[0] = -s; F->ew[1] = c; F->ew[2] = 0.0;
    F->eu[0] = c;  F->eu[1] = s; F->eu[2] = 0.0;
    F->ev[0] = 0;  F->ev[1] = 0; F->ev[2] = 1.0;
}

/* Unit direction from the source to the centre of pixel (iu, iv). */
static void ray_dir(const ocb* cb, const oframe* F, int iu, int iv, double dh[3]) {
    double u = (iu - 0.5 * (cb->nu - 1)) * cb->du + cb->off_u;
    double v = (iv - 0.5 * (cb->nv - 1)) * cb->dv + cb->off_v;
    double P[3], d[3], len = 0;
    for (int c = 0; c < 3; c++) {
        P[c] = F->S[c] + cb->sdd * F->ew[c] + u * F->eu[c] + v * F->ev[c];
        d[c] = P[c] - F->S[c];
        len += d[c] * d[c];
    }
    len = sqrt(len);
    for (int c = 0; c < 3; c++) dh[c] = d[c] / len;
}

/* Sample i of the ray, in voxel units: q = (S + i*step*dh - o) / s. */
static void sample_point(const ovol* vol, const oframe* F, const double dh[3], double step,
                         long i, double q[3]) {
    double o[3] = {vol->ox, vol->oy, vol->oz}, s[3] = {vol->sx, vol->sy, vol->sz};
    for (int c = 0; c < 3; c++) q[c] = (F->S[c] + (double)i * step * dh[c] - o[c]) / s[c];
}

/* A sample belongs to the ray sum when it lies in the support box [-1, n_c]
 * of the zero-padded trilinear interpolant. */
static int in_support(const ovol* vol, const double q[3]) {
    int n[3] = {vol->nx, vol->ny, vol->nz};
    for (int c = 0; c < 3; c++)
        if (q[c] < -1.0 || q[c] > (double)n[c]) return 0;
    return 1;
}

/* Candidate index range [i0, i1] of samples, from the slab intersection of the
 * ray with the support box, widened by one on each side; every candidate is
 * re-tested with in_support, so the range only needs to contain the set. */
static int sample_range(const ovol* vol, const oframe* F, const double dh[3], double step,
                        long* i0, long* i1) {
    double o[3] = {vol->ox, vol->oy, vol->oz}, s[3] = {vol->sx, vol->sy, vol->sz};
    int n[3] = {vol->nx, vol->ny, vol->nz};
    double tlo = -INFINITY, thi = INFINITY;
    for (int c = 0; c < 3; c++) {
        double lo = o[c] - s[c], hi = o[c] + n[c] * s[c]; /* world extent of [-1, n] */
        if (dh[c] == 0.0) {
            if (F->S[c] < lo || F->S[c] > hi) return 0;
            continue;
        }
        double t1 = (lo - F->S[c]) / dh[c], t2 = (hi - F->S[c]) / dh[c];
        if (t1 > t2) { double t = t1; t1 = t2; t2 = t; }
        if (t1 > tlo) tlo = t1;
        if (t2 < thi) thi = t2;
    }
    if (tlo > thi) return 0;
    *i0 = (long)ceil(tlo / step) - 1;
    *i1 = (long)floor(thi / step) + 1;
    return 1;
}

/* Every sample must lie ahead of the source (t > 0): require the whole
 * support box [-1, n_c] to sit in the half-space in front of it, measured
 * along the central ray direction ew (d . ew > 0 for every ray). */
static int box_in_front(const ovol* vol, const ocb* cb) {
    oframe F;
    view_frame(cb, &F);
    double o[3] = {vol->ox, vol->oy, vol->oz}, s[3] = {vol->sx, vol->sy, vol->sz};
    int n[3] = {vol->nx, vol->ny, vol->nz};
    for (int corner = 0; corner < 8; corner++) {
        double dot = 0;
        for (int c = 0; c < 3; c++) {
            double X = (corner >> c & 1) ? o[c] + n[c] * s[c] : o[c] - s[c];
            dot += (X - F.S[c]) * F.ew[c];
        }
        if (!(dot > 0)) return 0;
    }
    return 1;
}

static int cb_ok(const ovol* vol, const ocb* cb, double step) {
    return cb && cb->nu > 0 && cb->nv > 0 && cb->sad > 0 && cb->sdd > 0 && cb->du > 0 &&
           cb->dv > 0 && step > 0 && box_in_front(vol, cb);
}

/* --------------------------------------------------- projector P (Eq. 2) */
double oracle_drr_ray(const double* f, const ovol* vol, const ocb* cb, double step, int iu,
                      int iv) {
    oframe F;
    double dh[3], q[3], sum = 0.0;
    long i0, i1;
    view_frame(cb, &F);
    ray_dir(cb, &F, iu, iv, dh);
    if (!sample_range(vol, &F, dh, step, &i0, &i1)) return 0.0;
    for (long i = i0; i <= i1; i++) {
        sample_point(vol, &F, dh, step, i, q);
        if (in_support(vol, q)) sum += oracle_trilinear(f, vol, q[0], q[1], q[2]);
    }
    return step * sum;
}

int oracle_drr_forward(const double* f, const ovol* vol, const ocb* cb, double step, double* p) {
    if (!vol_ok(vol) || !cb_ok(vol, cb, step) || !f || !p) return 1;
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int iv = 0; iv < cb->nv; iv++)
        for (int iu = 0; iu < cb->nu; iu++)
            p[(long)iv * cb->nu + iu] = oracle_drr_ray(f, vol, cb, step, iu, iv);
    return 0;
}

/* ----------------------------------------- Siddon projector (Sec. II.B) */
static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

double oracle_siddon_ray(const double* f, const ovol* vol, const ocb* cb, int iu, int iv) {
    oframe F;
    double dh[3];
    view_frame(cb, &F);
    ray_dir(cb, &F, iu, iv, dh);
    double o[3] = {vol->ox, vol->oy, vol->oz}, s[3] = {vol->sx, vol->sy, vol->sz};
    int n[3] = {vol->nx, vol->ny, vol->nz};
    /* the ray's parameter interval inside the union of the voxel cubes */
    double tin = 0.0, tout = INFINITY;
    for (int c = 0; c < 3; c++) {
        double lo = o[c] - 0.5 * s[c], hi = o[c] + (n[c] - 0.5) * s[c];
        if (dh[c] == 0.0) {
            if (F.S[c] < lo || F.S[c] > hi) return 0.0;
            continue;
        }
        double t1 = (lo - F.S[c]) / dh[c], t2 = (hi - F.S[c]) / dh[c];
        if (t1 > t2) { double t = t1; t1 = t2; t2 = t; }
        if (t1 > tin) tin = t1;
        if (t2 < tout) tout = t2;
    }
    if (!(tin < tout)) return 0.0;
    /* every crossing with a voxel face plane inside (tin, tout), plus the ends */
    long cap = 2 + (long)(n[0] + 1) + (n[1] + 1) + (n[2] + 1);
    double* t = (double*)malloc(sizeof(double) * cap);
    long m = 0;
    t[m++] = tin;
    t[m++] = tout;
    for (int c = 0; c < 3; c++) {
        if (dh[c] == 0.0) continue;
        for (int l = 0; l <= n[c]; l++) {
            double tc = (o[c] + (l - 0.5) * s[c] - F.S[c]) / dh[c];
            if (tc > tin && tc < tout) t[m++] = tc;
        }
    }
    qsort(t, m, sizeof(double), cmp_double);
    double sum = 0.0;
    for (long e = 0; e + 1 < m; e++) {
        double len = t[e + 1] - t[e];
        if (!(len > 0.0)) continue;
        double tm = 0.5 * (t[e] + t[e + 1]);
        long idx[3];
        int inside = 1;
        for (int c = 0; c < 3; c++) {
            idx[c] = (long)floor((F.S[c] + tm * dh[c] - o[c]) / s[c] + 0.5);
            if (idx[c] < 0 || idx[c] >= n[c]) inside = 0;
        }
        if (inside) sum += len * f[(idx[2] * n[1] + idx[1]) * n[0] + idx[0]];
    }
    free(t);
    return sum;
}

int oracle_siddon_forward(const double* f, const ovol* vol, const ocb* cb, double* p) {
    if (!vol_ok(vol) || !cb_ok(vol, cb, 1.0) || !f || !p) return 1;
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int iv = 0; iv < cb->nv; iv++)
        for (int iu = 0; iu < cb->nu; iu++)
            p[(long)iv * cb->nu + iu] = oracle_siddon_ray(f, vol, cb, iu, iv);
    return 0;
}

/* P^T: for every (ray, sample) pair of P, add step * img(ray) * weight to the
 * eight taps of the sample -- the transpose of the sum in oracle_drr_ray. */
int oracle_drr_adjoint(const double* img, const ovol* vol, const ocb* cb, double step, double* g) {
    if (!vol_ok(vol) || !cb_ok(vol, cb, step) || !img || !g) return 1;
    long N = nvox(vol);
    memset(g, 0, sizeof(double) * N);
    oframe F;
    view_frame(cb, &F);
    for (int iv = 0; iv < cb->nv; iv++)
        for (int iu = 0; iu < cb->nu; iu++) {
            double r = img[(long)iv * cb->nu + iu], dh[3], q[3];
            long i0, i1;
            ray_dir(cb, &F, iu, iv, dh);
            if (r == 0.0 || !sample_range(vol, &F, dh, step, &i0, &i1)) continue;
            for (long i = i0; i <= i1; i++) {
                sample_point(vol, &F, dh, step, i, q);
                if (!in_support(vol, q)) continue;
                double fl = floor(q[0]), fm = floor(q[1]), fn = floor(q[2]);
                long l = (long)fl, m = (long)fm, n = (long)fn;
                double z[3] = {q[0] - fl, q[1] - fm, q[2] - fn};
                for (int t = 0; t < 8; t++) {
                    int a = t & 1, b = (t >> 1) & 1, c = (t >> 2) & 1;
                    long ii = l + a, jj = m + b, kk = n + c;
                    if (ii < 0 || jj < 0 || kk < 0 || ii >= vol->nx || jj >= vol->ny ||
                        kk >= vol->nz)
                        continue;
                    double wgt = (a ? z[0] : 1 - z[0]) * (b ? z[1] : 1 - z[1]) *
                                 (c ? z[2] : 1 - z[2]);
                    g[(kk * vol->ny + jj) * vol->nx + ii] += step * r * wgt;
                }
            }
        }
    return 0;
}

/* ---------------------------------------------------------------- Eq. (A.1)
 * (a, b)^T = (Y^T Y)^-1 Y^T p with Y = [y, 1]. */
int oracle_intensity_fit(const double* p, const double* y, long M, double* a, double* b) {
    if (!p || !y || M < 2) return 1;
    double Sy = 0, Syy = 0, Sp = 0, Syp = 0;
    for (long i = 0; i < M; i++) {
        Sy += y[i];
        Syy += y[i] * y[i];
        Sp += p[i];
        Syp += y[i] * p[i];
    }
    double det = (double)M * Syy - Sy * Sy;
    if (!(Syy > 0) || !(det > 1e-12 * (double)M * Syy)) return 2;
    *a = ((double)M * Syp - Sy * Sp) / det;
    *b = (Syy * Sp - Sy * Syp) / det;
    return 0;
}

/* ------------------------------------------------------------------ Eq. (2) */
double oracle_cost(const double* p, const double* y, long M, double a, double b) {
    double J = 0;
    for (long i = 0; i < M; i++) {
        double r = p[i] - a * y[i] - b;
        J += r * r;
    }
    return J;
}

/* Render p(w) = P f(w); f and dvf are caller scratch of N and 3N doubles. */
static int render(const double* f0, const double* mean, const double* U, int K, const double* w,
                  const ovol* vol, const ocb* cb, double step, double* dvf, double* f, double* p) {
    int st = oracle_pca_dvf(mean, U, K, w, vol, dvf);
    if (!st) st = oracle_warp_volume(f0, dvf, vol, f);
    if (!st) st = oracle_drr_forward(f, vol, cb, step, p);
    return st;
}

/* Gradient below Eq. (A.2): G = 2 U^T (df/dx) P^T r, with df/dx_c = (df/dq_c)/s_c
 * because q_c = idx_c + x_c / s_c. */
static void grad_from_residual(const double* f0, const double* U, int K, const double* dvf,
                               const double* g, const ovol* vol, double* G) {
    long N = nvox(vol);
    double s[3] = {vol->sx, vol->sy, vol->sz};
    for (int k = 0; k < K; k++) G[k] = 0;
    for (long kk = 0; kk < vol->nz; kk++)
        for (long j = 0; j < vol->ny; j++)
            for (long i = 0; i < vol->nx; i++) {
                long n = (kk * vol->ny + j) * vol->nx + i;
                if (g[n] == 0.0) continue;
                double d[3];
                oracle_trilinear_grad(f0, vol, i + dvf[n] / s[0], j + dvf[N + n] / s[1],
                                      kk + dvf[2 * N + n] / s[2], d);
                for (int k = 0; k < K; k++) {
                    double h = 0;
                    for (int c = 0; c < 3; c++) h += d[c] / s[c] * U[((long)k * 3 + c) * N + n];
                    G[k] += 2.0 * g[n] * h;
                }
            }
}

int oracle_cost_grad(const double* f0, const double* mean, const double* U, int K,
                     const double* w, const double* y, const ovol* vol, const ocb* cb,
                     double step, int fit_ab, double* ab, double* J, double* G) {
    if (!vol_ok(vol) || !cb_ok(vol, cb, step) || K < 1 || !f0 || !U || !w || !y || !ab)
        return 1;
    long N = nvox(vol), M = (long)cb->nu * cb->nv;
    double* dvf = malloc(sizeof(double) * 3 * N);
    double* f = malloc(sizeof(double) * N);
    double* g = malloc(sizeof(double) * N);
    double* p = malloc(sizeof(double) * M);
    double* r = malloc(sizeof(double) * M);
    int st = render(f0, mean, U, K, w, vol, cb, step, dvf, f, p);
    if (!st && fit_ab) st = oracle_intensity_fit(p, y, M, &ab[0], &ab[1]);
    if (!st) {
        *J = oracle_cost(p, y, M, ab[0], ab[1]);
        for (long i = 0; i < M; i++) r[i] = p[i] - ab[0] * y[i] - ab[1];
        st = oracle_drr_adjoint(r, vol, cb, step, g);
    }
    if (!st && G) grad_from_residual(f0, U, K, dvf, g, vol, G);
    free(dvf); free(f); free(g); free(p); free(r);
    return st;
}

int oracle_grad_forward_mode(const double* f0, const double* mean, const double* U, int K,
                             const double* w, const double* y, const ovol* vol,
                             const ocb* cb, double step, double a, double b, double* G) {
    if (!vol_ok(vol) || !cb_ok(vol, cb, step) || K < 1) return 1;
    long N = nvox(vol), M = (long)cb->nu * cb->nv;
    double s[3] = {vol->sx, vol->sy, vol->sz};
    double* dvf = malloc(sizeof(double) * 3 * N);
    double* f = malloc(sizeof(double) * N);
    double* h = malloc(sizeof(double) * N);
    double* p = malloc(sizeof(double) * M);
    double* ph = malloc(sizeof(double) * M);
    int st = render(f0, mean, U, K, w, vol, cb, step, dvf, f, p);
    for (int k = 0; !st && k < K; k++) {
#pragma omp parallel for schedule(static)
        for (long kk = 0; kk < vol->nz; kk++)
            for (long j = 0; j < vol->ny; j++)
                for (long i = 0; i < vol->nx; i++) {
                    long n = (kk * vol->ny + j) * vol->nx + i;
                    double d[3];
                    oracle_trilinear_grad(f0, vol, i + dvf[n] / s[0], j + dvf[N + n] / s[1],
                                          kk + dvf[2 * N + n] / s[2], d);
                    double hv = 0;
                    for (int c = 0; c < 3; c++) hv += d[c] / s[c] * U[((long)k * 3 + c) * N + n];
                    h[n] = hv;
                }
        st = oracle_drr_forward(h, vol, cb, step, ph);
        double acc = 0;
        for (long i = 0; i < M; i++) acc += (p[i] - a * y[i] - b) * ph[i];
        G[k] = 2.0 * acc;
    }
    free(dvf); free(f); free(h); free(p); free(ph);
    return st;
}


/* ------------------------------------------------- warp transpose (W^T)
 * The warp is linear in f0: f(v) = sum over the eight taps u of q(v) of
 * weight(q(v), u) f0(u), with taps outside the grid dropped.  Its transpose
 * scatters z(v) with the same weights. */
int oracle_warp_adjoint(const double* z, const double* dvf, const ovol* vol, double* out) {
    if (!vol_ok(vol) || !z || !dvf || !out) return 1;
    long N = nvox(vol);
    memset(out, 0, sizeof(double) * N);
    for (long k = 0; k < vol->nz; k++)
        for (long j = 0; j < vol->ny; j++)
            for (long i = 0; i < vol->nx; i++) {
                long n = (k * vol->ny + j) * vol->nx + i;
                double q[3] = {i + dvf[n] / vol->sx, j + dvf[N + n] / vol->sy, k + dvf[2 * N + n] / vol->sz};
                double fl[3] = {floor(q[0]), floor(q[1]), floor(q[2])};
                double zz[3] = {q[0] - fl[0], q[1] - fl[1], q[2] - fl[2]};
                for (int t = 0; t < 8; t++) {
                    int a = t & 1, b = (t >> 1) & 1, cc = (t >> 2) & 1;
                    long ii = (long)fl[0] + a, jj = (long)fl[1] + b, kk = (long)fl[2] + cc;
                    if (ii < 0 || jj < 0 || kk < 0 || ii >= vol->nx || jj >= vol->ny || kk >= vol->nz)
                        continue;
                    double wgt = (a ? zz[0] : 1 - zz[0]) * (b ? zz[1] : 1 - zz[1]) * (cc ? zz[2] : 1 - zz[2]);
                    out[(kk * vol->ny + jj) * vol->nx + ii] += wgt * z[n];
                }
            }
    return 0;
}

int oracle_cost_grad_f0(const double* f0, const double* mean, const double* U, int K,
                        const double* w, const double* y, const ovol* vol, const ocb* cb,
                        double step, int fit_ab, double* ab, double* J, double* dJdf0) {
    if (!vol_ok(vol) || !cb_ok(vol, cb, step) || K < 1 || !f0 || !U || !w || !y || !ab || !J || !dJdf0)
        return 1;
    long N = nvox(vol), M = (long)cb->nu * cb->nv;
    double* dvf = malloc(sizeof(double) * 3 * N);
    double* f = malloc(sizeof(double) * N);
    double* g = malloc(sizeof(double) * N);
    double* p = malloc(sizeof(double) * M);
    double* r = malloc(sizeof(double) * M);
    int st = render(f0, mean, U, K, w, vol, cb, step, dvf, f, p);
    if (!st && fit_ab) st = oracle_intensity_fit(p, y, M, &ab[0], &ab[1]);
    if (!st) {
        *J = oracle_cost(p, y, M, ab[0], ab[1]);
        for (long i = 0; i < M; i++) r[i] = 2.0 * (p[i] - ab[0] * y[i] - ab[1]);   /* dJ/dp */
        st = oracle_drr_adjoint(r, vol, cb, step, g);                              /* dJ/df */
    }
    if (!st) st = oracle_warp_adjoint(g, dvf, vol, dJdf0);                         /* dJ/df0 */
    free(dvf); free(f); free(g); free(p); free(r);
    return st;
}

/* ------------------------------------------------- Appendix: the alternating solve
 * Each iteration: (A.1) refits (a, b) on the current projection; the gradient
 * at fixed (a, b) gives d = -G/||G||; Armijo backtracking from mu0 accepts the
 * first mu with J(w + mu d) <= J(w) - alpha mu ||G||, else mu <- beta mu.  When
 * mu drops below mu_min (or the trial cap is reached) no step is taken and the
 * solve stops; it also stops after max_iter iterations or when ||G|| = 0. */
int oracle_solve_projection_log(const double* f0, const double* mean, const double* U, int K,
                                const double* y, const ovol* vol, const ocb* cb,
                                const double* w_init, const oparams* prm, double* w_out,
                                ostats* st, double* J_trace, double* it_log) {
    if (!vol_ok(vol) || !prm || !cb_ok(vol, cb, prm->step) || K < 1 || K > 64 || !w_init ||
        !w_out || !st)
        return 1;
    long N = nvox(vol), M = (long)cb->nu * cb->nv;
    double step = prm->step;
    double* dvf = malloc(sizeof(double) * 3 * N);
    double* f = malloc(sizeof(double) * N);
    double* g = malloc(sizeof(double) * N);
    double* p = malloc(sizeof(double) * M);
    double* pt = malloc(sizeof(double) * M);
    double* r = malloc(sizeof(double) * M);
    double w[64], wt[64], d[64], G[64];
    int rc = 0;
    memset(st, 0, sizeof(*st));
    for (int k = 0; k < K; k++) w[k] = w_init[k];
    rc = render(f0, mean, U, K, w, vol, cb, step, dvf, f, p);
    st->evals = 1;
    double a = 0, b = 0, J = 0, mu = prm->mu0;
    for (int it = 0; !rc && it < prm->max_iter; it++) {
        rc = oracle_intensity_fit(p, y, M, &a, &b);            /* step 1, (A.1) */
        if (rc) break;
        J = oracle_cost(p, y, M, a, b);
        if (it == 0) st->J0 = J;
        if (J_trace) J_trace[it] = J;
        const double Jw = J;
        double wlog[64];
        for (int k = 0; k < K; k++) wlog[k] = w[k];
        /* gradient at w with (a, b) fixed; dvf/f currently hold w's fields */
        rc = oracle_pca_dvf(mean, U, K, w, vol, dvf);
        for (long i = 0; i < M; i++) r[i] = p[i] - a * y[i] - b;
        if (!rc) rc = oracle_drr_adjoint(r, vol, cb, step, g);
        if (rc) break;
        grad_from_residual(f0, U, K, dvf, g, vol, G);
        double gn = 0;
        for (int k = 0; k < K; k++) gn += G[k] * G[k];
        gn = sqrt(gn);
        if (gn == 0.0) break;
        for (int k = 0; k < K; k++) d[k] = -G[k] / gn;
        int accepted = 0, tried = 0;
        mu = prm->mu0;                                            /* step 2, (A.2) */
        for (int tr = 0; tr < prm->max_trials && mu >= prm->mu_min; tr++) {
            tried++;
            for (int k = 0; k < K; k++) wt[k] = w[k] + mu * d[k];
            rc = render(f0, mean, U, K, wt, vol, cb, step, dvf, f, pt);
            st->evals++;
            if (rc) break;
            double Jt = oracle_cost(pt, y, M, a, b);
            if (Jt <= J - prm->alpha * mu * gn) {
                for (int k = 0; k < K; k++) w[k] = wt[k];
                double* tmp = p; p = pt; pt = tmp;
                J = Jt;
                accepted = 1;
                break;
            }
            mu *= prm->beta;
        }
        if (rc) break;
        if (it_log) {
            double* row = it_log + (long)it * ORACLE_LOG_STRIDE(K);
            row[0] = Jw; row[1] = a; row[2] = b; row[3] = gn;
            row[4] = accepted ? mu : 0.0; row[5] = tried; row[6] = accepted;
            for (int k = 0; k < K; k++) {
                row[7 + k] = wlog[k];
                row[7 + K + k] = G[k];
                row[7 + 2 * K + k] = d[k];
            }
        }
        st->iters++;
        if (J_trace) J_trace[it + 1] = J;
        if (!accepted) break;
    }
    st->J = J; st->a = a; st->b = b; st->mu_last = mu; st->status = rc;
    for (int k = 0; k < K; k++) w_out[k] = w[k];
    free(dvf); free(f); free(g); free(p); free(pt); free(r);
    return rc;
}

int oracle_solve_projection(const double* f0, const double* mean, const double* U, int K,
                            const double* y, const ovol* vol, const ocb* cb,
                            const double* w_init, const oparams* prm, double* w_out,
                            ostats* st, double* J_trace) {
    return oracle_solve_projection_log(f0, mean, U, K, y, vol, cb, w_init, prm, w_out, st, J_trace, NULL);
}

/* ------------------------------------------------- Sec. II.A: localisation
 * The DVF x is a pull-back field: the new-image point c maps to c + x(c) in
 * the reference image.  The tumour position c solves c + x(c) = c_ref; with
 * c = c_ref + y the fixed point is y = -x(c_ref + y) (Chen et al., ref. 18). */
static void dvf_at_point(const double* mean, const double* U, int K, const double* w,
                         const ovol* vol, const double X[3], double x[3]) {
    long N = nvox(vol);
    double q1 = (X[0] - vol->ox) / vol->sx, q2 = (X[1] - vol->oy) / vol->sy,
           q3 = (X[2] - vol->oz) / vol->sz;
    for (int c = 0; c < 3; c++) {
        double v = mean ? oracle_trilinear(mean + c * N, vol, q1, q2, q3) : 0.0;
        for (int k = 0; k < K; k++)
            v += w[k] * oracle_trilinear(U + ((long)k * 3 + c) * N, vol, q1, q2, q3);
        x[c] = v;
    }
}

int oracle_localize_tumor(const double* mean, const double* U, int K, const double* w,
                          const ovol* vol, const double c_ref[3], int max_iter,
                          double tol_mm, double c_out[3]) {
    if (!vol_ok(vol) || K < 0 || !c_ref || !c_out || max_iter < 1) return 1;
    double y[3] = {0, 0, 0};
    int converged = 0;
    for (int it = 0; it < max_iter; it++) {
        double X[3] = {c_ref[0] + y[0], c_ref[1] + y[1], c_ref[2] + y[2]}, x[3];
        dvf_at_point(mean, U, K, w, vol, X, x);
        double ch = 0;
        for (int c = 0; c < 3; c++) {
            double yn = -x[c];
            ch = fmax(ch, fabs(yn - y[c]));
            y[c] = yn;
        }
        if (ch < tol_mm) { converged = 1; break; }
    }
    for (int c = 0; c < 3; c++) c_out[c] = c_ref[c] + y[c];
    return converged ? 0 : 4;
}

/* ------------------------------------------------------------------ Eq. (3)
 * For each coefficient k separately, least squares over t = L..T-1 of
 * trace[t][k] ~ sum_l c_kl trace[t-l][k]; solved by the normal equations with
 * Gaussian elimination and partial pivoting. */
int oracle_lp_fit(const double* trace, int T, int K, int L, double* c) {
    if (!trace || !c || K < 1 || L < 1 || L > 16 || T <= 2 * L) return 1;
    for (int k = 0; k < K; k++) {
        double A[16][17];
        memset(A, 0, sizeof(A));
        for (int t = L; t < T; t++) {
            for (int i = 0; i < L; i++) {
                double xi = trace[(long)(t - 1 - i) * K + k];
                for (int j = 0; j < L; j++) A[i][j] += xi * trace[(long)(t - 1 - j) * K + k];
                A[i][L] += xi * trace[(long)t * K + k];
            }
        }
        for (int col = 0; col < L; col++) {
            int piv = col;
            for (int i = col + 1; i < L; i++)
                if (fabs(A[i][col]) > fabs(A[piv][col])) piv = i;
            if (A[piv][col] == 0.0) return 2;
            if (piv != col)
                for (int j = 0; j <= L; j++) { double t = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = t; }
            for (int i = col + 1; i < L; i++) {
                double fct = A[i][col] / A[col][col];
                for (int j = col; j <= L; j++) A[i][j] -= fct * A[col][j];
            }
        }
        for (int i = L - 1; i >= 0; i--) {
            double s = A[i][L];
            for (int j = i + 1; j < L; j++) s -= A[i][j] * c[k * L + j];
            c[k * L + i] = s / A[i][i];
        }
    }
    return 0;
}

int oracle_lp_predict(const double* hist, const double* c, int K, int L, double* w0) {
    if (!hist || !c || !w0 || K < 1 || L < 1) return 1;
    for (int k = 0; k < K; k++) {
        double s = 0;
        for (int l = 1; l <= L; l++) s += c[k * L + (l - 1)] * hist[(long)(l - 1) * K + k];
        w0[k] = s;
    }
    return 0;
}
