// pcas_internal.cuh -- device-side types and helpers shared by the CUDA
// translation units of libpcasolve (sm_103a).  Not part of the C ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

#include "pcasolve.h"

namespace pcas {

// ----------------------------------------------------------------- geometry
// One cone-beam view expressed in voxel units of the volume (q = (X - o) / s).
// Ray of pixel (iu, iv): world direction d = sdd ew + u eu + v ev with
// u = u0 + iu du, v = v0 + iv dv; since ew, eu, ev are orthonormal,
// |d|^2 = sdd^2 + u^2 + v^2.  In voxel units D = (A + u Bu + v Bv) / |d|.
struct View {
    float3 Q0;               // source position (S - o) / s
    float3 A, Bu, Bv;        // sdd ew / s, eu / s, ev / s
    float3 EW, EU, EV;       // s * ew, s * eu, s * ev (voxel offsets -> mm along the axes)
    float sdd, sdd2;
    float u0, du, v0, dv;    // detector coordinates of pixel centres, mm
    int nu, nv;
    float step;              // ray-march step, mm
    int swap;                // layout of the solver volumes: 1 = x and y exchanged
                             // (see solver_pad), chosen per angle
    int lw1, lw4;            // projector warp patches (ray_pixel), chosen per angle
    int chunk1, chunk4;      // projector chunks (ray_sums_staged), chosen per angle
    // Fixed-view cache of P^T (null: the gather computes the weights): per
    // voxel (world index) its footprint on the detector and, from an offset in
    // floats, the weight of every ray of that rectangle, row by row.
    const short4* pt_rect;   // iu0, iv0, iu1, iv1 (empty when iu0 > iu1 or iv0 > iv1)
    const unsigned long long* pt_off;
    const float* pt_w;
};

struct Grid {
    int nx, ny, nz;
    float inv_sx, inv_sy, inv_sz;
};

// Internal warped-volume layout with a zero halo two voxels deep: voxel
// (i,j,k) lives at element ((k+2) pny + (j+2)) px + (i+4).  px is a multiple of
// 4 and >= nx + 6, so interior rows start 16-byte aligned, and every tap of a
// sample within half a voxel of the support box [-1, n] lands inside the
// allocation on a halo zero or a voxel: the ray march needs no clamps.
struct Pad {
    int px, pny, pnz;
};

__host__ __device__ inline Pad make_pad(int nx, int ny, int nz) {
    Pad p;
    p.px = ((nx + 6) + 3) & ~3;
    p.pny = ny + 4;
    p.pnz = nz + 4;
    return p;
}

__host__ __device__ inline long pad_index(const Pad& pd, int i, int j, int k) {
    return ((long)(k + 2) * pd.pny + (j + 2)) * pd.px + (i + 4);
}

// Solver volume layout.  A warp's rays are neighbours along the detector u
// axis, which is world x at gantry 0 and world y at 90 degrees, so which
// voxels they read together depends on the angle.  Each solver volume is
// stored either x fastest or with x and y exchanged (y fastest), chosen per
// 22.5-degree bin of the angle (Tune); the projector then marches the
// mirrored geometry: the same sample points with x and y exchanged.
__host__ __device__ inline Pad solver_pad(int nx, int ny, int nz, int xy_swap) {
    return xy_swap ? make_pad(ny, nx, nz) : make_pad(nx, ny, nz);
}

// Trial step sizes evaluated together in one warp + projection pass: the
// first four interleaved as float4 in the candidate buffer, the fifth in the
// one-volume buffer (free during a batch).  Five covers the whole default
// schedule mu0, beta mu0, ..., beta^4 mu0 >= mu_min of an iteration.
enum { TRIAL_BATCH = 5, NBUF = TRIAL_BATCH + 1 };

// ----------------------------------------------------------- solver state
enum Phase : int {
    PH_RUNNING = 0,     // a trial is pending
    PH_ACCEPT = 1,      // the last trial passed the Armijo test
    PH_STOP = 2,        // no mu >= mu_min passed: iteration counted, solve ends
    PH_ZERO_GRAD = 3,   // ||G|| = 0: solve ends before the line search
    PH_SINGULAR = 4     // Y^T Y singular in Eq. (A.1)
};

enum { NMOM = 6 };      // Sp, Syp, Spp, Srr, Sy, Syy

struct SolveState {
    double w[PCAS_KMAX], d[PCAS_KMAX], G[PCAS_KMAX];
    double wt[TRIAL_BATCH][PCAS_KMAX];    // candidate coefficients w + mu_j d of the batch
    double mu_batch[TRIAL_BATCH];         // their step sizes, in the backtracking order
    double gnorm, a, b, J, J0, Jt, mu;
    double mom[NBUF][NMOM];               // final moments of the projection buffers
    double mu0, alpha, beta, mu_min;
    int K, max_trials;
    int cur;                              // buffer holding P f(w)
    int phase, evals, trials;
    int nvalid;                           // candidates of the pending batch still on the schedule
    int wide;                             // 0: the last iteration took its first step size, so the
                                          // next iteration's first batch renders two candidates
    int iters, batches;                   // device-driven solve: completed iterations, batches this iteration
    int max_iter, launches;               // launches: kernels run by a device-driven solve
    unsigned int counter[4];              // last-block counters (reset by the last block)
    // Bounding box of the non-zero voxels of the warped volume (slot 0: f,
    // slot 1: the union of the batch's candidates), as {xmin, ymin, zmin, -xmax,
    // -ymax, -zmax} so that both ends reduce with atomicMin; "empty" is
    // BOX_EMPTY everywhere.  Written by the warp kernels, read and reset by the
    // projector that consumes the volume.
    int box[2][6];
    unsigned int occ_gen;                 // pass number of the occupancy bricks (never reset)
    int keep_f0h;                         // device-driven run: the halo copy of f0 is current
    int jac_ready;                        // the first evaluation's warp did the next gradient's
                                          // Jacobian pass (launch_warp_jac); its gather clears it
};

enum : int { BOX_EMPTY = 0x3fffffff };

// ------------------------------------------------------ occupancy bricks
// Empty-space skipping of the solver projectors (exact), on bricks of B^3
// voxels, B = 1 << OCC_LOG = 4.  A sample of the march whose cell has its
// (0,0,0) tap at c = floor(q) (frame voxel indices) belongs to brick
// ((c_x + 1) >> OCC_LOG, ...), clamped to the grid of (n >> OCC_LOG) + 1
// bricks per axis; its eight taps lie in [B b - 1, B b + B - 1] per axis.
// (The bricks bound each ray's samples to the span between its first and
// last occupied brick, so smaller bricks cut the empty samples at the ends
// of the span: about 8 % of the samples with B = 8, 4 % with B = 4 on the
// sequence phantom.)  The warp kernels mark every brick whose taps
// include a non-zero voxel of the volumes they write with the current pass
// number; the projector that reads those volumes treats a brick holding any
// other number as empty: each of its samples interpolates eight zero taps and
// adds exactly +0, so leaving such samples out of a ray changes no bit of the
// sum.  Marks of earlier passes can only make the projector do more work, so
// the mask is never cleared; the projector's last block advances the number.
// The reference CT has bricks of its own (8^3 voxels, world axes, one byte
// each, 0 or 1; f0b_n): k_fill_f0h marks them when it writes the halo copy,
// and the warp and Jacobian kernels interpolate only in cells of marked
// bricks -- elsewhere all eight taps are zero and so is the result (A.5) and
// its gradient (A.8).
struct Occ {
    unsigned int* mask;       // null: no marking and no skipping
    unsigned int* gen;        // the pass number (SolveState::occ_gen)
    const unsigned char* f0m; // bricks of the reference CT (null: none)
};
constexpr int OCC_LOG = 2;
__host__ __device__ inline int occ_n(int n) { return (n >> OCC_LOG) + 1; }
__host__ __device__ inline long occ_count(int nx, int ny, int nz) {
    return (long)occ_n(nx) * occ_n(ny) * occ_n(nz);
}
// Bricks of the reference CT (8^3 voxels).
__host__ __device__ inline int f0b_n(int n) { return (n >> 3) + 1; }
__host__ __device__ inline long f0b_count(int nx, int ny, int nz) {
    return (long)f0b_n(nx) * f0b_n(ny) * f0b_n(nz);
}
// Occupancy bricks of the solver frame (see Occ): the frame exchanges x and y
// when swp is set.
struct OccFrame {
    unsigned int* m;
    unsigned int gen;
    int nbx, nby;
};
__device__ __forceinline__ OccFrame occ_frame(const Occ& oc, int nx, int ny, int swp) {
    OccFrame o{oc.mask, 0u, occ_n(swp ? ny : nx), occ_n(swp ? nx : ny)};
    if (oc.mask) o.gen = *oc.gen;
    return o;
}
// Marks the bricks whose taps include a frame voxel of [x0, x1] x [y0, y1] x
// {z}: voxel v is a tap of the cells of bricks v >> OCC_LOG and
// (v + 1) >> OCC_LOG along each axis (two bricks where v + 1 is a multiple
// of B).
__device__ __forceinline__ void occ_mark(unsigned int* m, unsigned int gen, int nbx, int nby, int x0, int x1,
                                         int y0, int y1, int z) {
    for (int bz = z >> OCC_LOG; bz <= (z + 1) >> OCC_LOG; bz++)
        for (int by = y0 >> OCC_LOG; by <= (y1 + 1) >> OCC_LOG; by++)
            for (int bx = x0 >> OCC_LOG; bx <= (x1 + 1) >> OCC_LOG; bx++) m[((long)bz * nby + by) * nbx + bx] = gen;
}

// Number of the next (up to TRIAL_BATCH) step sizes mu, beta mu, ... that the
// backtracking rule may still try: mu >= mu_min and fewer than max_trials
// trials in this iteration.  The host mirrors the same loop.
__host__ __device__ inline int count_valid(double mu, double beta, double mu_min, int trials, int max_trials) {
    int n = 0;
    while (n < TRIAL_BATCH && mu >= mu_min && trials + n < max_trials) {
        n++;
        mu *= beta;
    }
    return n;
}

// Reduction scratch: per-block partials plus the counter used to find the
// last block to finish (which then reduces all partials in a fixed order).
struct Reduce {
    double* part;
    unsigned int* counter;
};

// ------------------------------------------------------ storage types
// The reference CT and the motion model may be stored as float, bfloat16 or
// half; every value is widened to float on load (interpolation, DVF synthesis
// and accumulation are float).
template <typename T> __device__ __forceinline__ float ldg_f(const T* p);
template <> __device__ __forceinline__ float ldg_f<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ldg_f<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ float ldg_f<__half>(const __half* p) { return __half2float(__ldg(p)); }

// Four consecutive values, streaming (evict-first); p 16-byte (float) or
// 8-byte (16-bit types) aligned.
template <typename T> __device__ __forceinline__ float4 ld4_stream(const T* p);
template <> __device__ __forceinline__ float4 ld4_stream<float>(const float* p) {
    return __ldcs(reinterpret_cast<const float4*>(p));
}
template <> __device__ __forceinline__ float4 ld4_stream<__nv_bfloat16>(const __nv_bfloat16* p) {
    const uint2 u = __ldcs(reinterpret_cast<const uint2*>(p));
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
}
template <> __device__ __forceinline__ float4 ld4_stream<__half>(const __half* p) {
    const uint2 u = __ldcs(reinterpret_cast<const uint2*>(p));
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
template <typename T> __device__ __forceinline__ float ldcs_f(const T* p);
template <> __device__ __forceinline__ float ldcs_f<float>(const float* p) { return __ldcs(p); }
template <> __device__ __forceinline__ float ldcs_f<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(__ldcs(p));
}
template <> __device__ __forceinline__ float ldcs_f<__half>(const __half* p) { return __half2float(__ldcs(p)); }

// ------------------------------------------------------------- trilinear
// Eq. (A.5): trilinear interpolation with zero outside the grid, on the dense
// [nz][ny][nx] layout.  Positions are clamped to [-2, n+1] first so that
// conversion to int is always defined (values there are zero anyway).
template <typename T>
__device__ __forceinline__ float tri_dense(const T* __restrict__ f, const Grid& g,
                                           float qx, float qy, float qz) {
    qx = fminf(fmaxf(qx, -2.0f), (float)g.nx + 1.0f);
    qy = fminf(fmaxf(qy, -2.0f), (float)g.ny + 1.0f);
    qz = fminf(fmaxf(qz, -2.0f), (float)g.nz + 1.0f);
    float fx = floorf(qx), fy = floorf(qy), fz = floorf(qz);
    int lx = (int)fx, ly = (int)fy, lz = (int)fz;
    float zx = qx - fx, zy = qy - fy, zz = qz - fz;
    const int sy = g.nx, sz = g.nx * g.ny;    // 32-bit offsets: volumes have < 2^31 voxels
    float v000, v100, v010, v110, v001, v101, v011, v111;
    // interior cell (all eight taps in the grid): 0 <= l < n - 1 per axis, as one unsigned compare
    if ((unsigned)lx < (unsigned)(g.nx - 1) && (unsigned)ly < (unsigned)(g.ny - 1) &&
        (unsigned)lz < (unsigned)(g.nz - 1)) {
        const T* b = f + lz * sz + ly * sy + lx;
        v000 = ldg_f(b);           v100 = ldg_f(b + 1);
        v010 = ldg_f(b + sy);      v110 = ldg_f(b + sy + 1);
        v001 = ldg_f(b + sz);      v101 = ldg_f(b + sz + 1);
        v011 = ldg_f(b + sz + sy); v111 = ldg_f(b + sz + sy + 1);
    } else {
        const bool x0 = lx >= 0 && lx < g.nx, x1 = lx + 1 >= 0 && lx + 1 < g.nx;
        const bool y0 = ly >= 0 && ly < g.ny, y1 = ly + 1 >= 0 && ly + 1 < g.ny;
        const bool z0 = lz >= 0 && lz < g.nz, z1 = lz + 1 >= 0 && lz + 1 < g.nz;
        auto at = [&](bool ok, int i, int j, int k) -> float {
            return ok ? ldg_f(f + k * sz + j * sy + i) : 0.0f;
        };
        v000 = at(x0 && y0 && z0, lx, ly, lz);
        v100 = at(x1 && y0 && z0, lx + 1, ly, lz);
        v010 = at(x0 && y1 && z0, lx, ly + 1, lz);
        v110 = at(x1 && y1 && z0, lx + 1, ly + 1, lz);
        v001 = at(x0 && y0 && z1, lx, ly, lz + 1);
        v101 = at(x1 && y0 && z1, lx + 1, ly, lz + 1);
        v011 = at(x0 && y1 && z1, lx, ly + 1, lz + 1);
        v111 = at(x1 && y1 && z1, lx + 1, ly + 1, lz + 1);
    }
    float c00 = fmaf(zx, v100 - v000, v000), c10 = fmaf(zx, v110 - v010, v010);
    float c01 = fmaf(zx, v101 - v001, v001), c11 = fmaf(zx, v111 - v011, v011);
    float c0 = fmaf(zy, c10 - c00, c00), c1 = fmaf(zy, c11 - c01, c01);
    return fmaf(zz, c1 - c0, c0);
}

// The reference CT as the solver kernels read it: float, with a zero halo
// three voxels deep (voxel (i,j,k) at ((k+3)(ny+6) + (j+3))(nx+6) + (i+3)).
// With positions clamped to [-2, n+1] as tri_dense does, all eight taps are
// in the allocation and are exactly the zero-padded values tri_dense reads:
// the same interpolant, bit for bit, without per-tap tests.
enum { F0_HALO = 3 };
__host__ __device__ inline long f0h_count(int nx, int ny, int nz) {
    return (long)(nx + 2 * F0_HALO) * (ny + 2 * F0_HALO) * (nz + 2 * F0_HALO);
}

// The eight taps of the cell holding q (tap t = dx + 2 dy + 4 dz) and the
// fractions, from the halo copy.
__device__ __forceinline__ void taps_halo(const float* __restrict__ f, const Grid& g, float qx, float qy,
                                          float qz, float v[8], float& zx, float& zy, float& zz) {
    qx = fminf(fmaxf(qx, -2.0f), (float)g.nx + 1.0f);
    qy = fminf(fmaxf(qy, -2.0f), (float)g.ny + 1.0f);
    qz = fminf(fmaxf(qz, -2.0f), (float)g.nz + 1.0f);
    const float fx = floorf(qx), fy = floorf(qy), fz = floorf(qz);
    zx = qx - fx; zy = qy - fy; zz = qz - fz;
    const int sy = g.nx + 2 * F0_HALO, sz = sy * (g.ny + 2 * F0_HALO);
    const float* b = f + (((int)fz + F0_HALO) * sz + ((int)fy + F0_HALO) * sy + ((int)fx + F0_HALO));
    v[0] = __ldg(b);           v[1] = __ldg(b + 1);
    v[2] = __ldg(b + sy);      v[3] = __ldg(b + sy + 1);
    v[4] = __ldg(b + sz);      v[5] = __ldg(b + sz + 1);
    v[6] = __ldg(b + sz + sy); v[7] = __ldg(b + sz + sy + 1);
}

// tri_halo for a position already inside the clamp range [-2, n + 1] of every
// axis (the clamps would not change it): the same taps and arithmetic.
__device__ __forceinline__ float tri_halo_in(const float* __restrict__ f, const Grid& g, float qx, float qy,
                                             float qz) {
    const float fx = floorf(qx), fy = floorf(qy), fz = floorf(qz);
    const float zx = qx - fx, zy = qy - fy, zz = qz - fz;
    const int sy = g.nx + 2 * F0_HALO, sz = sy * (g.ny + 2 * F0_HALO);
    const float* b = f + (((int)fz + F0_HALO) * sz + ((int)fy + F0_HALO) * sy + ((int)fx + F0_HALO));
    const float v0 = __ldg(b), v1 = __ldg(b + 1), v2 = __ldg(b + sy), v3 = __ldg(b + sy + 1);
    const float v4 = __ldg(b + sz), v5 = __ldg(b + sz + 1), v6 = __ldg(b + sz + sy), v7 = __ldg(b + sz + sy + 1);
    const float c00 = fmaf(zx, v1 - v0, v0), c10 = fmaf(zx, v3 - v2, v2);
    const float c01 = fmaf(zx, v5 - v4, v4), c11 = fmaf(zx, v7 - v6, v6);
    const float c0 = fmaf(zy, c10 - c00, c00), c1 = fmaf(zy, c11 - c01, c01);
    return fmaf(zz, c1 - c0, c0);
}

// Brick of the reference CT holding the cell that taps_halo takes at q
// (world axes, the same clamps and floors), as an index into its mask.
__device__ __forceinline__ int f0_brick(const Grid& g, float qx, float qy, float qz) {
    qx = fminf(fmaxf(qx, -2.0f), (float)g.nx + 1.0f);
    qy = fminf(fmaxf(qy, -2.0f), (float)g.ny + 1.0f);
    qz = fminf(fmaxf(qz, -2.0f), (float)g.nz + 1.0f);
    const int nbx = f0b_n(g.nx), nby = f0b_n(g.ny), nbz = f0b_n(g.nz);
    const int bx = min(max(((int)floorf(qx) + 1) >> 3, 0), nbx - 1);
    const int by = min(max(((int)floorf(qy) + 1) >> 3, 0), nby - 1);
    const int bz = min(max(((int)floorf(qz) + 1) >> 3, 0), nbz - 1);
    return (bz * nby + by) * nbx + bx;
}

// Eq. (A.5) from the halo copy: tri_dense's result without its branches.
__device__ __forceinline__ float tri_halo(const float* __restrict__ f, const Grid& g, float qx, float qy,
                                          float qz) {
    float v[8], zx, zy, zz;
    taps_halo(f, g, qx, qy, qz, v, zx, zy, zz);
    const float c00 = fmaf(zx, v[1] - v[0], v[0]), c10 = fmaf(zx, v[3] - v[2], v[2]);
    const float c01 = fmaf(zx, v[5] - v[4], v[4]), c11 = fmaf(zx, v[7] - v[6], v[6]);
    const float c0 = fmaf(zy, c10 - c00, c00), c1 = fmaf(zy, c11 - c01, c01);
    return fmaf(zz, c1 - c0, c0);
}

// Whether any cell taps_halo may take for a position in the box [lo, hi]
// (per axis) lies in a marked brick of the reference CT (m: its bricks).
// The clamped brick coordinate is monotone in the position, so the cells of
// the box's positions lie in the bricks between those of its corners; a box
// spanning more than two bricks along an axis is reported live.
__device__ __forceinline__ bool f0_box_live(const unsigned char* __restrict__ m, const Grid& g, float lox,
                                            float loy, float loz, float hix, float hiy, float hiz) {
    const int nbx = f0b_n(g.nx), nby = f0b_n(g.ny), nbz = f0b_n(g.nz);
    auto br = [](float q, int n, int nb) {
        q = fminf(fmaxf(q, -2.0f), (float)n + 1.0f);
        return min(max(((int)floorf(q) + 1) >> 3, 0), nb - 1);
    };
    const int x0 = br(lox, g.nx, nbx), x1 = br(hix, g.nx, nbx);
    const int y0 = br(loy, g.ny, nby), y1 = br(hiy, g.ny, nby);
    const int z0 = br(loz, g.nz, nbz), z1 = br(hiz, g.nz, nbz);
    if (x1 - x0 > 1 || y1 - y0 > 1 || z1 - z0 > 1) return true;
    for (int z = z0; z <= z1; z++)
        for (int y = y0; y <= y1; y++)
            for (int x = x0; x <= x1; x++)
                if (__ldg(m + (z * nby + y) * nbx + x)) return true;
    return false;
}

// tri_halo, or +0 without touching the taps when the cell's brick of the
// reference CT is empty (m: its bricks, or null).  The same bits either way.
__device__ __forceinline__ float tri_halo_m(const float* __restrict__ f, const unsigned char* __restrict__ m,
                                            const Grid& g, float qx, float qy, float qz) {
    if (m && !__ldg(m + f0_brick(g, qx, qy, qz))) return 0.0f;
    return tri_halo(f, g, qx, qy, qz);
}

__device__ __forceinline__ float lerp1(float z, float a, float b) { return fmaf(z, b - a, a); }
__device__ __forceinline__ float4 lerp4(float z, const float4& a, const float4& b) {
    return make_float4(lerp1(z, a.x, b.x), lerp1(z, a.y, b.y), lerp1(z, a.z, b.z), lerp1(z, a.w, b.w));
}

// Four interleaved volumes (one float4 per voxel) sampled at the same point:
// the weights are computed once, the eight taps are 16-byte loads.
__device__ __forceinline__ float4 tri_padded4(const float4* __restrict__ f, const Pad& pd, float qx,
                                              float qy, float qz) {
    const float fx = floorf(qx), fy = floorf(qy), fz = floorf(qz);
    const float zx = qx - fx, zy = qy - fy, zz = qz - fz;
    const int sy = pd.px, sz = pd.px * pd.pny;
    const float4* b = f + (((int)fz + 2) * sz + ((int)fy + 2) * sy + ((int)fx + 4));
    const float4 c00 = lerp4(zx, __ldg(b), __ldg(b + 1));
    const float4 c10 = lerp4(zx, __ldg(b + sy), __ldg(b + sy + 1));
    const float4 c01 = lerp4(zx, __ldg(b + sz), __ldg(b + sz + 1));
    const float4 c11 = lerp4(zx, __ldg(b + sz + sy), __ldg(b + sz + sy + 1));
    return lerp4(zz, lerp4(zy, c00, c10), lerp4(zy, c01, c11));
}

// Same interpolant on the zero-halo layout (Pad), read from its x-pair copy:
// element e holds (f[e], f[e + 1]) of the layout (zero where either lies in
// the halo), so the eight taps are four 8-byte loads.  No bounds tests and no
// clamps: valid for q within half a voxel of [-1, n] (the caller guarantees
// it), where the floor is in [-2, n] and every tap is a voxel or a halo zero.
__device__ __forceinline__ float tri_padded_pairs(const float2* __restrict__ f, const Pad& pd, float qx,
                                                  float qy, float qz) {
    const float fx = floorf(qx), fy = floorf(qy), fz = floorf(qz);
    const float zx = qx - fx, zy = qy - fy, zz = qz - fz;
    const int sy = pd.px, sz = pd.px * pd.pny;
    const float2* b = f + (((int)fz + 2) * sz + ((int)fy + 2) * sy + ((int)fx + 4));
    const float2 p00 = __ldg(b), p10 = __ldg(b + sy), p01 = __ldg(b + sz), p11 = __ldg(b + sz + sy);
    const float c00 = fmaf(zx, p00.y - p00.x, p00.x), c10 = fmaf(zx, p10.y - p10.x, p10.x);
    const float c01 = fmaf(zx, p01.y - p01.x, p01.x), c11 = fmaf(zx, p11.y - p11.x, p11.x);
    const float c0 = fmaf(zy, c10 - c00, c00), c1 = fmaf(zy, c11 - c01, c01);
    return fmaf(zz, c1 - c0, c0);
}

// ----------------------------------------------------------------- rays
template <typename X>
__device__ __forceinline__ void swap_xy(X& a, X& b) { X t = a; a = b; b = t; }

// The view, grid and layout of a solver volume in the frame it is stored in
// (see solver_pad): a no-op unless swap is set.
__device__ __forceinline__ void solver_frame(View& V, Grid& g, Pad& pd, int swap) {
    if (swap) {
        swap_xy(V.Q0.x, V.Q0.y); swap_xy(V.A.x, V.A.y); swap_xy(V.Bu.x, V.Bu.y); swap_xy(V.Bv.x, V.Bv.y);
        swap_xy(V.EW.x, V.EW.y); swap_xy(V.EU.x, V.EU.y); swap_xy(V.EV.x, V.EV.y);
        swap_xy(g.nx, g.ny); swap_xy(g.inv_sx, g.inv_sy);
    }
    pd = make_pad(g.nx, g.ny, g.nz);
}

// Unit ray direction of pixel (iu, iv) in voxel units per mm.  Every
// operation is explicit (no contraction left to the compiler), so each kernel
// that calls it gets the same bits for a ray.
__device__ __forceinline__ float3 ray_dir(const View& V, int iu, int iv) {
    float u = fmaf((float)iu, V.du, V.u0), v = fmaf((float)iv, V.dv, V.v0);
    float inv = 1.0f / sqrtf(fmaf(v, v, fmaf(u, u, V.sdd2)));
    float3 D;
    D.x = fmaf(u, V.Bu.x, fmaf(v, V.Bv.x, V.A.x)) * inv;
    D.y = fmaf(u, V.Bu.y, fmaf(v, V.Bv.y, V.A.y)) * inv;
    D.z = fmaf(u, V.Bu.z, fmaf(v, V.Bv.z, V.A.z)) * inv;
    return D;
}

// Range [i0, i1] of sample indices whose position Q0 + i step D lies in the
// box [lo_c, hi_c] (voxel units); empty when i0 > i1.  Rounding can add or
// drop a sample right on the box surface, where the interpolant is zero.
__device__ __forceinline__ void sample_range_box(const View& V, float3 D, const float lo[3],
                                                 const float hi[3], int& i0, int& i1) {
    float tlo = -3.0e38f, thi = 3.0e38f;
    const float q0[3] = {V.Q0.x, V.Q0.y, V.Q0.z};
    const float d[3] = {D.x, D.y, D.z};
#pragma unroll
    for (int c = 0; c < 3; c++) {
        if (d[c] != 0.0f) {
            float ia = 1.0f / d[c];
            float t1 = (lo[c] - q0[c]) * ia, t2 = (hi[c] - q0[c]) * ia;
            tlo = fmaxf(tlo, fminf(t1, t2));
            thi = fminf(thi, fmaxf(t1, t2));
        } else if (q0[c] < lo[c] || q0[c] > hi[c]) {
            tlo = 1.0f; thi = 0.0f;
        }
    }
    if (!(tlo <= thi)) { i0 = 1; i1 = 0; return; }
    i0 = (int)ceilf(tlo / V.step);
    i1 = (int)floorf(thi / V.step);
}

// The support box [-1, n_c] of the zero-padded trilinear interpolant.
__device__ __forceinline__ void sample_range(const View& V, const Grid& g, float3 D, int& i0,
                                             int& i1) {
    const float lo[3] = {-1.0f, -1.0f, -1.0f};
    const float hi[3] = {(float)g.nx, (float)g.ny, (float)g.nz};
    sample_range_box(V, D, lo, hi, i0, i1);
}

// --------------------------------------------------------------- reductions
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-level reduction of NV per-thread float values: FP32 inside each warp,
// FP64 across warps.  Writes this block's NV doubles to red.part[blk * NV + j]
// and returns true in every thread of the block that finished last; that
// block's thread j < NV then holds the fixed-order FP64 total in out[j]
// (shared memory).  blockDim.x must be a multiple of 32, at most 32 NW.
template <int NV, int NW = 32>
__device__ bool block_reduce_last(const float (&v)[NV], Reduce red, unsigned int nblocks,
                                  unsigned int blk, double* out /* shared, NV */) {
    __shared__ double s_w[NW][NV];      // per-warp sums; reused for the final tree
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; j++) {
        float t = warp_sum(v[j]);
        if (lane == 0) s_w[wid][j] = (double)t;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < nw; w++) s += s_w[w][threadIdx.x];
        red.part[(size_t)blk * NV + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int prev = atomicAdd(red.counter, 1u);
        s_last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    // fixed-order reduction: thread t sums blocks t, t+nt, ...; then a tree
    double(&s_acc)[NW][NV] = s_w;      // free again: read before the barriers above
    double acc[NV];
#pragma unroll
    for (int j = 0; j < NV; j++) acc[j] = 0.0;
    for (unsigned int b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
        for (int j = 0; j < NV; j++) acc[j] += __ldcg(red.part + (size_t)b * NV + j);
    }
#pragma unroll
    for (int j = 0; j < NV; j++) {
        double t = warp_sum_d(acc[j]);
        if (lane == 0) s_acc[wid][j] = t;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < nw; w++) s += s_acc[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
    if (threadIdx.x == 0) *red.counter = 0u;
    __syncthreads();
    return true;
}

// ------------------------------------------------------------ launch shapes
// Launch shapes of the solver kernels, chosen per size bucket: the defaults
// below, or the ones pcas_autotune measured fastest for the bucket.
enum { NBIN = 8 };            // 22.5-degree bins of the gantry angle modulo 180 degrees
struct Tune {
    int lw1;                  // log2 of a warp's patch width in pixels along u (2..4) of the
                              // one-volume projector; the patch is (1 << lw) x (32 >> lw),
                              // four warps per block stacked along v
    int chunk1;               // sample indices per staged chunk of the one-volume projector;
                              // 0: it marches through L1 (no staging)
    int vt;                   // voxel tile of the gradient pass (vox_tile)
    int adj_mult;             // gather blocks per SM
    int skip;                 // empty-space skipping of the projectors (occupancy bricks)
    unsigned char lw4[NBIN];      // per angle bin: patch width of the batch projector,
    unsigned char chunk4[NBIN];   // its staged chunk,
    unsigned char swap[NBIN];     // and the layout of the solver volumes (solver_pad)
};

// Voxel tiles of the gradient pass (256 voxels): log2 of the x, y, z extents.
enum { NVOXTILE = 6 };
__host__ __device__ inline void vox_tile(int vt, int& lx, int& ly, int& lz) {
    switch (vt) {
        case 1: lx = 4; ly = 2; lz = 2; break;   // 16 x 4 x 4
        case 2: lx = 5; ly = 2; lz = 1; break;   // 32 x 4 x 2
        case 3: lx = 4; ly = 3; lz = 1; break;   // 16 x 8 x 2
        case 4: lx = 5; ly = 3; lz = 0; break;   // 32 x 8 x 1
        case 5: lx = 6; ly = 2; lz = 0; break;   // 64 x 4 x 1
        default: lx = 3; ly = 3; lz = 2; break;  // 8 x 8 x 4
    }
}
inline long adj_tiles(int nx, int ny, int nz, int vt) {
    int lx, ly, lz;
    vox_tile(vt, lx, ly, lz);
    return (long)((nx + (1 << lx) - 1) >> lx) * ((ny + (1 << ly) - 1) >> ly) * ((nz + (1 << lz) - 1) >> lz);
}
inline long adj_tiles_max(int nx, int ny, int nz) {
    long m = 0;
    for (int vt = 0; vt < NVOXTILE; vt++) {
        const long t = adj_tiles(nx, ny, nz, vt);
        m = t > m ? t : m;
    }
    return m;
}

// Blocks of the solver projector for a patch width of 1 << lw pixels
// (blocks of 128 rays: (1 << lw) x (128 >> lw) pixels).  The solver launches
// drr_blocks(nu, nv) blocks, enough for every width; with the width read from
// the view, a block's index maps to (bx, by) = (blk % gx, blk / gx) and blocks
// past the detector have no rays.
inline unsigned drr_blocks_x(int nu, int lw) { return (unsigned)((nu + (1 << lw) - 1) >> lw); }
inline unsigned drr_blocks_y(int nv, int lw) { return (unsigned)((nv + (128 >> lw) - 1) / (128 >> lw)); }
inline unsigned drr_blocks(int nu, int nv) {           // the largest grid over lw = 2..4
    unsigned m = 0;
    for (int lw = 2; lw <= 4; lw++) {
        const unsigned b = drr_blocks_x(nu, lw) * drr_blocks_y(nv, lw);
        m = b > m ? b : m;
    }
    return m;
}

// ------------------------------------------------------- launch interfaces
struct WSrc {                 // where a PCA-model kernel takes w from
    float w[PCAS_KMAX];       // used when dev is null
    const double* dev;        // device w (solver state), K doubles
    const int* phase;         // early exit when *phase >= PH_STOP (may be null)
};

// Storage type of f0 / mean / U (values of pcas_dtype in pcasolve.h).
enum DType : int { DT_F32 = 0, DT_BF16 = 1, DT_F16 = 2 };

cudaError_t launch_pca_dvf(const void* mean, const void* U, int dt, int K, const float* w, Grid g,
                           float* dvf, cudaStream_t s);
cudaError_t launch_warp_dvf(const void* f0, int dt, const float* dvf, Grid g, float* f, cudaStream_t s);
// Copies f0 (storage type dt) into the interior of the halo copy f0h (whose
// halo the caller has zeroed; it is never written).
// f0m (may be null): bricks of the reference CT, zeroed by the caller, marked here.
// skip (device, may be null): the copy is skipped while *skip is non-zero.
cudaError_t launch_fill_f0h(const void* f0, int dt, Grid g, float* f0h, unsigned char* f0m, const int* skip,
                            cudaStream_t s);
// Solver warps: launch_warp_pca writes f(w_src) to the scalar zero-halo
// buffer fpad, or, when fpair is not null, to fpair as x pairs (see
// tri_padded_pairs) and not to fpad; launch_warp_batch writes the batch:
// candidates st->wt[0..3] interleaved (float4) and wt[4] to fpad.
// Vd (device, may be null): its swap selects the layout (solver_pad); the
// bounding box is recorded in the same frame.
// f0h: the halo copy of the reference CT (float); mean and U in storage type dt.
// oc: occupancy bricks of the written volumes (oc.mask null: none).
cudaError_t launch_warp_pca(const float* f0h, const void* mean, const void* U, int dt, int K, WSrc w,
                            Grid g, const View* Vd, float* fpad, float2* fpair, int* box, Occ oc, cudaStream_t s);
cudaError_t launch_warp_batch(const float* f0h, const void* mean, const void* U, int dt, int K,
                              const SolveState* st, Grid g, const View* Vd, float4* fpad4, float* fpad,
                              Occ oc, cudaStream_t s);
cudaError_t launch_drr_plain(const float* f, Grid g, const View& V, float* p, cudaStream_t s);
// Siddon geometry in double precision (world mm): source, unit axes, pixel
// grid and the voxel grid (origin = centre of voxel (0,0,0)).
struct SidView {
    double S[3], ew[3], eu[3], ev[3];
    double sdd, u0, du, v0, dv;
    double o[3], s[3];
    int n[3], nu, nv;
};
cudaError_t launch_drr_siddon(const float* f, const SidView& V, float* p, cudaStream_t s);
// Solver projector.  mode 0: first evaluation into buffer cur;
// mode TRIAL_BATCH: the five-volume batch (st->nvalid of them on the
// schedule).  Vh: the view on the host (grid size), Vd: the same in device
// memory (read by the kernels, so captured launches stay view-independent).
// hbatch / use_h: inside a device-driven solve the batch projector sets this
// conditional handle to whether another candidate batch follows.  oc: the
// occupancy bricks the warp kernels marked for these volumes (oc.mask null:
// every ray keeps its box-clipped range).  Mode 0 reads the x pairs fpair
// when T.chunk1 is 0 (the march through L1) and fpad when it stages chunks.
cudaError_t launch_drr_solver(const float* fpad, const float2* fpair, const float4* fpad4, Grid g,
                              const View& Vh, const View* Vd, const float* y, float* pbuf, int mode,
                              SolveState* st, double* part, const Tune& T, unsigned long long hbatch,
                              int use_h, Occ oc, cudaStream_t s);
cudaError_t launch_resid(const float* pbuf, const float* y, const View& Vh, const View* Vd, int first,
                         float4* rayt, SolveState* st, double* part, cudaStream_t s);
cudaError_t launch_adjoint_plain(const float* img, Grid g, const View& V, float* gout,
                                 cudaStream_t s);
// Scratch of the gradient pass: compacted voxels with a non-zero warp
// Jacobian (place in the voxel tile and h_k, per tile of 256) and the tile
// counts / offsets.
struct AdjScratch {
    int* act_idx;       // ntiles * 256
    float* act_h;       // K * ntiles * 256
    int* tile_count;    // ntiles
    int* tile_off;      // ntiles + 1
};
// The first evaluation's warp fused with the Jacobian pass of the gradient at
// the same w: one read of the motion model gives f(w), written as
// launch_warp_pca writes it (fpad, or its x-pair copy fpair when not null;
// bounding box into box, occupancy bricks of the output in occ), and the
// compacted voxels of the gradient pass in voxel tile vt, as its Jacobian pass
// writes them; the next launch_adjoint_grad (same vt) then skips its Jacobian
// pass (SolveState::jac_ready).  view: its swap selects the layout.
struct JacWarp {
    const View* view;
    float* fpad;
    float2* fpair;
    int* box;
    Occ occ;
};
cudaError_t launch_warp_jac(Grid g, const float* f0h, const unsigned char* f0m, const void* mean, const void* U,
                            int dt, int K, SolveState* st, const AdjScratch& as, int vt, const JacWarp& jw,
                            cudaStream_t s);
// hbatch / use_h: inside a device-driven solve the gradient's last block opens
// (or not) the iteration's candidate-batch loop by setting this handle.
// join (may be null): an event the gather waits for (the residual pass, which
// the Jacobian pass does not need, can then run beside it on another stream).
// f0m (may be null): bricks of the reference CT (see Occ).
cudaError_t launch_adjoint_grad(const float4* rayt, Grid g, const View* V, const float* f0h,
                                const unsigned char* f0m, const void* mean, const void* U, int dt, int K,
                                int step_setup,
                                SolveState* st, double* part, const AdjScratch& as, int vt, int max_blocks,
                                unsigned long long hbatch, int use_h, cudaEvent_t join, cudaStream_t s);
// dJ/df0 = W^T (2 P^T r): z (N floats) and acc (N 64-bit) are scratch,
// zmax_bits one word; out (N floats) receives the gradient.
cudaError_t launch_grad_f0(const float4* rayt, Grid g, const View* V, const float* mean, const float* U,
                           int K, const SolveState* st, float* z, unsigned int* zmax_bits,
                           unsigned long long* acc, float* out, cudaStream_t s);
cudaError_t launch_localize(const float* mean, const float* U, int K, const double* w, Grid g,
                            const double o[3], const double s_mm[3], const double c_ref[3],
                            int max_iter, double tol, double* out, cudaStream_t s);

// Fixed-view P^T cache (View::pt_*): footprint sizes of every voxel (world
// order) into area, their exclusive scan into off (may be null) with the total
// into *total, and the footprints and weights themselves (err set when a
// footprint does not fit its slot, off[n + 1] - off[n]).
cudaError_t launch_pt_count(const View& V, Grid g, unsigned int* area, cudaStream_t s);
cudaError_t launch_pt_scan(const unsigned int* area, long n, unsigned long long* off, unsigned long long* total,
                           cudaStream_t s);
cudaError_t launch_pt_build(const View& V, Grid g, const unsigned long long* off, short4* rect, float* w, int* err,
                            cudaStream_t s);

// Number of partial slots each solver kernel needs (sizes the workspace).
enum { DRR_PART_VALS = 4 * TRIAL_BATCH + 2 };   // per-volume Sp, Syp, Spp, Srr + Sy, Syy
inline unsigned resid_blocks(int nu, int nv) { return (unsigned)(((long)nu * nv + 255) / 256); }
enum { ADJ_MAX_BLOCKS = 4096 };

}  // namespace pcas
