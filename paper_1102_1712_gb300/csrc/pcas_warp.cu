// pcas_warp.cu -- DVF synthesis (Eq. 1) fused into the trilinear warp of the
// reference CT (Eq. A.3/A.5).  HBM-bound: the motion model (12 (K+1) bytes per
// voxel) streams once per evaluation with 16-byte loads and evict-first
// policy, f0 is gathered through L1/L2, and f is written once.
#include "pcas_internal.cuh"

namespace pcas {
namespace {

constexpr int kWarpThreads = 256;
constexpr int kBatchVPT = 4;     // voxels per thread of the batch warp

// Eq. (1) on four consecutive voxels: x_c = mean_c + sum_k w_k U_kc.
template <typename T>
__device__ __forceinline__ void dvf4(const T* __restrict__ mean, const T* __restrict__ U,
                                     int K, const float* w, long N, long n, float x[3][4]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        float4 m = mean ? ld4_stream(mean + c * N + n) : make_float4(0.f, 0.f, 0.f, 0.f);
        x[c][0] = m.x; x[c][1] = m.y; x[c][2] = m.z; x[c][3] = m.w;
    }
    for (int k = 0; k < K; k++) {
        const float wk = w[k];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            float4 u = ld4_stream(U + ((long)k * 3 + c) * N + n);
            x[c][0] = fmaf(wk, u.x, x[c][0]);
            x[c][1] = fmaf(wk, u.y, x[c][1]);
            x[c][2] = fmaf(wk, u.z, x[c][2]);
            x[c][3] = fmaf(wk, u.w, x[c][3]);
        }
    }
}

// Bounding box of the non-zero outputs of a block (thread-local boxes reduced
// through warp shuffles, then one atomicMin per component and block): both
// reductions are order-independent, so the box is deterministic.
__device__ __forceinline__ void box_reduce(int b[6], int* __restrict__ out) {
    __shared__ int s_b[kWarpThreads / 32][6];
#pragma unroll
    for (int t = 0; t < 6; t++)
        for (int o = 16; o > 0; o >>= 1) b[t] = min(b[t], __shfl_xor_sync(0xffffffffu, b[t], o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        for (int t = 0; t < 6; t++) s_b[wid][t] = b[t];
    __syncthreads();
    if (threadIdx.x < 6) {
        int m = BOX_EMPTY;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = min(m, s_b[w][threadIdx.x]);
        if (m != BOX_EMPTY) atomicMin(out + threadIdx.x, m);
    }
}

__device__ __forceinline__ void box_add(int b[6], int i, int j, int k) {
    b[0] = min(b[0], i); b[1] = min(b[1], j); b[2] = min(b[2], k);
    b[3] = min(b[3], -i); b[4] = min(b[4], -j); b[5] = min(b[5], -k);
}

// Eq. (1) alone: dvf = mean + U w.  One thread per 4 voxels (VEC) or 1 voxel.
template <bool VEC, typename T>
__global__ void __launch_bounds__(kWarpThreads)
k_pca_dvf(const T* __restrict__ mean, const T* __restrict__ U, int K, WSrc ws, long N,
          float* __restrict__ dvf) {
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (VEC) {
        long n = t * 4;
        if (n >= N) return;
        float x[3][4];
        dvf4(mean, U, K, ws.w, N, n, x);
#pragma unroll
        for (int c = 0; c < 3; c++)
            *reinterpret_cast<float4*>(dvf + c * N + n) = make_float4(x[c][0], x[c][1], x[c][2], x[c][3]);
    } else {
        if (t >= N) return;
        for (int c = 0; c < 3; c++) {
            float x = mean ? ldg_f(mean + c * N + t) : 0.0f;
            for (int k = 0; k < K; k++) x = fmaf(ws.w[k], ldg_f(U + ((long)k * 3 + c) * N + t), x);
            dvf[c * N + t] = x;
        }
    }
}

// Warp by an explicit DVF (public warp_volume): one voxel per thread, dense out.
template <typename T>
__global__ void __launch_bounds__(kWarpThreads)
k_warp_dvf(const T* __restrict__ f0, const float* __restrict__ dvf, Grid g, long N,
           float* __restrict__ f) {
    long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    int i = (int)(n % g.nx);
    long r = n / g.nx;
    int j = (int)(r % g.ny), k = (int)(r / g.ny);
    float qx = fmaf(dvf[n], g.inv_sx, (float)i);
    float qy = fmaf(dvf[N + n], g.inv_sy, (float)j);
    float qz = fmaf(dvf[2 * N + n], g.inv_sz, (float)k);
    f[n] = tri_dense(f0, g, qx, qy, qz);
}

// Thread layout of the solver warps: blockIdx.z = k, blockIdx.y = j and
// i = (blockIdx.x blockDim.x + threadIdx.x) V with V voxels per thread (no
// index divisions; 32-bit voxel offsets, volumes have < 2^31 voxels).

// The halo copy of the reference CT (see tri_halo): interior only.  With f0m
// it marks the bricks whose taps include a non-zero voxel (see Occ): voxel i
// is a tap of the cells of bricks i >> 3 and (i + 1) >> 3 along each axis;
// one lane per warp marks the span of the warp's non-zero voxels of a row.
// Blocks stride over the rows (j, k).  skip (may be null): when it holds a
// non-zero value the copy is current and the kernel returns at once.
template <typename T>
__global__ void __launch_bounds__(kWarpThreads)
k_fill_f0h(const T* __restrict__ f0, Grid g, float* __restrict__ f0h, unsigned char* __restrict__ f0m,
           const int* __restrict__ skip) {
    if (skip && *skip) return;
    const long sy = g.nx + 2 * F0_HALO, sz = sy * (g.ny + 2 * F0_HALO);
    const int nbx = f0b_n(g.nx), nby = f0b_n(g.ny);
    const int rows = g.ny * g.nz;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int j = r % g.ny, k = r / g.ny;
        for (int i0 = 0; i0 < g.nx; i0 += blockDim.x) {      // the same trip count for every lane
            const int i = i0 + threadIdx.x;
            float v = 0.0f;
            if (i < g.nx) {
                v = ldg_f(f0 + ((long)k * g.ny + j) * g.nx + i);
                f0h[(k + F0_HALO) * sz + (j + F0_HALO) * sy + (i + F0_HALO)] = v;
            }
            if (!f0m) continue;
            const int lo = __reduce_min_sync(0xffffffffu, v != 0.0f ? i : INT_MAX);
            const int hi = __reduce_max_sync(0xffffffffu, v != 0.0f ? i : INT_MIN);
            if ((threadIdx.x & 31) != 0 || lo > hi) continue;
            for (int bz = k >> 3; bz <= (k + 1) >> 3; bz++)
                for (int by = j >> 3; by <= (j + 1) >> 3; by++)
                    for (int bx = lo >> 3; bx <= (hi + 1) >> 3; bx++) f0m[(bz * nby + by) * nbx + bx] = 1;
        }
    }
}

// Fused DVF synthesis + warp into the zero-halo layout used by the solver
// (fpad), or into its x-pair copy (fpair not null: each voxel stored as the
// first value of its own pair and the second of the pair before it; the
// pairs' halo values stay the zeros the caller wrote); marks the occupancy
// bricks of its non-zero voxels.
// VEC: 4 voxels per thread along x (nx % 4 == 0, 16-byte aligned model).
template <bool VEC, typename T>
__global__ void __launch_bounds__(kWarpThreads)
k_warp_pca(const float* __restrict__ f0h, const T* __restrict__ mean,
           const T* __restrict__ U, int K, WSrc ws, Grid g, const View* __restrict__ Vp,
           float* __restrict__ fpad, float2* __restrict__ fpair, int* __restrict__ box_out, Occ occ) {
    if (ws.phase && *ws.phase >= PH_STOP) return;
    const int swp = Vp ? Vp->swap : 0;
    const Pad pd = solver_pad(g.nx, g.ny, g.nz, swp);
    const OccFrame oc = occ_frame(occ, g.nx, g.ny, swp);
    __shared__ float s_w[PCAS_KMAX];
    if (threadIdx.x < PCAS_KMAX) {
        float wv = 0.f;                     // static indices keep ws out of local memory
#pragma unroll
        for (int t = 0; t < PCAS_KMAX; t++)
            if (threadIdx.x == t) wv = ws.w[t];
        s_w[threadIdx.x] = ws.dev ? (threadIdx.x < K ? (float)ws.dev[threadIdx.x] : 0.f) : wv;
    }
    __syncthreads();
    int b[6] = {BOX_EMPTY, BOX_EMPTY, BOX_EMPTY, BOX_EMPTY, BOX_EMPTY, BOX_EMPTY};
    const int j = blockIdx.y, k = blockIdx.z;
    const long N = (long)g.nx * g.ny * g.nz;
    const int row = (k * g.ny + j) * g.nx;
    if (VEC) {
        const int i = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
        if (i < g.nx) {
            const int n = row + i;
            float x[3][4];
            dvf4(mean, U, K, s_w, N, n, x);
            float o[4];
            int e0 = 4, e1 = -1;                    // first and last non-zero of the four
#pragma unroll
            for (int e = 0; e < 4; e++) {
                o[e] = tri_halo_m(f0h, occ.f0m, g, fmaf(x[0][e], g.inv_sx, (float)(i + e)),
                                   fmaf(x[1][e], g.inv_sy, (float)j), fmaf(x[2][e], g.inv_sz, (float)k));
                if (o[e] != 0.0f) {
                    if (swp) box_add(b, j, i + e, k);
                    else box_add(b, i + e, j, k);
                    e0 = min(e0, e);
                    e1 = e;
                }
            }
            if (oc.m && e1 >= 0) {
                if (swp) occ_mark(oc.m, oc.gen, oc.nbx, oc.nby, j, j, i + e0, i + e1, k);
                else occ_mark(oc.m, oc.gen, oc.nbx, oc.nby, i + e0, i + e1, j, j, k);
            }
            if (fpair) {                    // voxel d is .x of pair d and .y of pair d - 1
                float* p = reinterpret_cast<float*>(fpair);
                if (swp) {
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const long d = pad_index(pd, j, i + e, k);
                        p[2 * d - 1] = o[e];
                        p[2 * d] = o[e];
                    }
                } else {                    // d a multiple of 4: floats 2d - 1 ... 2d + 6
                    const long d = pad_index(pd, i, j, k);
                    p[2 * d - 1] = o[0];
                    *reinterpret_cast<float4*>(p + 2 * d) = make_float4(o[0], o[1], o[1], o[2]);
                    *reinterpret_cast<float2*>(p + 2 * d + 4) = make_float2(o[2], o[3]);
                    p[2 * d + 6] = o[3];
                }
            } else if (swp) {
#pragma unroll
                for (int e = 0; e < 4; e++) fpad[pad_index(pd, j, i + e, k)] = o[e];
            } else {
                *reinterpret_cast<float4*>(fpad + pad_index(pd, i, j, k)) = make_float4(o[0], o[1], o[2], o[3]);
            }
        }
    } else {
        const int i = blockIdx.x * blockDim.x + threadIdx.x;
        if (i < g.nx) {
            const int n = row + i;
            float x[3];
            for (int c = 0; c < 3; c++) {
                float v = mean ? ldg_f(mean + c * N + n) : 0.0f;
                for (int kk = 0; kk < K; kk++) v = fmaf(s_w[kk], ldg_f(U + ((long)kk * 3 + c) * N + n), v);
                x[c] = v;
            }
            const float o = tri_halo_m(f0h, occ.f0m, g, fmaf(x[0], g.inv_sx, (float)i),
                                        fmaf(x[1], g.inv_sy, (float)j), fmaf(x[2], g.inv_sz, (float)k));
            const int a0 = swp ? j : i, a1 = swp ? i : j;
            if (o != 0.0f) {
                box_add(b, a0, a1, k);
                if (oc.m) occ_mark(oc.m, oc.gen, oc.nbx, oc.nby, a0, a0, a1, a1, k);
            }
            const long d = pad_index(pd, a0, a1, k);
            if (fpair) {
                float* p = reinterpret_cast<float*>(fpair);
                p[2 * d - 1] = o;
                p[2 * d] = o;
            } else {
                fpad[d] = o;
            }
        }
    }
    box_reduce(b, box_out);
}

// The five candidate volumes of a line-search batch at once (Eq. 1 + A.5 for
// each w + mu_j d): the motion model is read once per voxel and reused for the
// five coefficient vectors; each DVF is formed in the same operation order as
// the single-volume warp, so a candidate's volume is bit-identical to a lone
// evaluation.  Each thread takes VPT voxels of its row, blockDim.x apart.  Output: one float4 (f_0..f_3) per voxel in the candidate
// buffer and f_4 in the one-volume buffer, zero-halo layout; the occupancy
// bricks mark the union of the five.  All five are rendered even when fewer
// are on the schedule (a narrow batch projects only the first two): the
// kernel is issue-bound, and a run-time candidate count in it costs more
// than the gathers it would save.
template <typename T, int KT, int VPT>
__global__ void __launch_bounds__(kWarpThreads, KT <= 3 ? 6 : (KT <= 5 ? 5 : (KT <= 7 ? 4 : 3)))
k_warp_batch(const float* __restrict__ f0h, const T* __restrict__ mean,
             const T* __restrict__ U, const SolveState* st, Grid g, const View* __restrict__ Vp,
             float4* __restrict__ fpad4, float* __restrict__ fpad, int* __restrict__ box_out, Occ occ) {
    if (st->phase >= PH_STOP || st->nvalid < 1) return;    // same gate as the batch projector
    const int swp = Vp ? Vp->swap : 0;
    const Pad pd = solver_pad(g.nx, g.ny, g.nz, swp);
    const OccFrame oc = occ_frame(occ, g.nx, g.ny, swp);
    __shared__ float s_w[TRIAL_BATCH][KT];
    if (threadIdx.x < TRIAL_BATCH * KT) {
        const int j = threadIdx.x / KT, k = threadIdx.x % KT;
        s_w[j][k] = (float)st->wt[j][k];
    }
    __syncthreads();
    // read from shared memory at each use (broadcast), not kept in registers
    const volatile float(*wk)[KT] = s_w;
    // the block's voxels share j and k: of the output's bounding box only the
    // x extent varies within it
    int ilo = BOX_EMPTY, ihi = BOX_EMPTY;     // min i, min -i of the non-zero voxels
    const int j = blockIdx.y, k = blockIdx.z;
    const long N = (long)g.nx * g.ny * g.nz;
    // VPT voxels per thread, blockDim.x apart (each pass of the loop stores
    // coalesced rows): the per-thread set-up and the block's box reduction are
    // shared by them
#pragma unroll 1
    for (int r = 0; r < VPT; r++) {
        const int i = (blockIdx.x * VPT + r) * blockDim.x + threadIdx.x;
        if (i < g.nx) {
            const int n = (k * g.ny + j) * g.nx + i;
            float x[TRIAL_BATCH][3];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float m = mean ? ldcs_f(mean + c * N + n) : 0.0f;
#pragma unroll
                for (int b = 0; b < TRIAL_BATCH; b++) x[b][c] = m;
            }
            const T* u0 = U + n;
            float u[KT][3];
#pragma unroll
            for (int kk = 0; kk < KT; kk++)
#pragma unroll
                for (int c = 0; c < 3; c++) u[kk][c] = ldcs_f(u0 + (kk * 3 + c) * N);
#pragma unroll
            for (int kk = 0; kk < KT; kk++)      // Eq. (1) in the order of the single-volume warp
#pragma unroll
                for (int b = 0; b < TRIAL_BATCH; b++) {
                    const float wbk = wk[b][kk];
#pragma unroll
                    for (int c = 0; c < 3; c++) x[b][c] = fmaf(wbk, u[kk][c], x[b][c]);
                }
            float q[TRIAL_BATCH][3];
#pragma unroll
            for (int b = 0; b < TRIAL_BATCH; b++) {
                q[b][0] = fmaf(x[b][0], g.inv_sx, (float)i);
                q[b][1] = fmaf(x[b][1], g.inv_sy, (float)j);
                q[b][2] = fmaf(x[b][2], g.inv_sz, (float)k);
            }
            // the box of the five positions: one brick test for all of them
            // (when every brick their cells can lie in is empty, all eight taps
            // of each are zero and so are the candidates), and inside the
            // grid's clamp range [-2, n + 1] the taps are read without clamps
            float lo[3], hi[3];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                lo[c] = hi[c] = q[0][c];
#pragma unroll
                for (int b = 1; b < TRIAL_BATCH; b++) {
                    lo[c] = fminf(lo[c], q[b][c]);
                    hi[c] = fmaxf(hi[c], q[b][c]);
                }
            }
            const bool live = !occ.f0m || f0_box_live(occ.f0m, g, lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]);
            const bool inside = lo[0] >= -2.0f && lo[1] >= -2.0f && lo[2] >= -2.0f && hi[0] <= (float)g.nx + 1.0f &&
                                hi[1] <= (float)g.ny + 1.0f && hi[2] <= (float)g.nz + 1.0f;
            float o[TRIAL_BATCH];
#pragma unroll
            for (int b = 0; b < TRIAL_BATCH; b++) o[b] = 0.0f;
            if (live && inside) {
#pragma unroll
                for (int b = 0; b < TRIAL_BATCH; b++) o[b] = tri_halo_in(f0h, g, q[b][0], q[b][1], q[b][2]);
            } else if (live) {
#pragma unroll
                for (int b = 0; b < TRIAL_BATCH; b++) o[b] = tri_halo(f0h, g, q[b][0], q[b][1], q[b][2]);
            }
            const int a0 = swp ? j : i, a1 = swp ? i : j;
            const long d = pad_index(pd, a0, a1, k);
            fpad4[d] = make_float4(o[0], o[1], o[2], o[3]);
            fpad[d] = o[4];
            if (o[0] != 0.0f || o[1] != 0.0f || o[2] != 0.0f || o[3] != 0.0f || o[4] != 0.0f) {
                ilo = min(ilo, i);
                ihi = min(ihi, -i);
                if (oc.m) occ_mark(oc.m, oc.gen, oc.nbx, oc.nby, a0, a0, a1, a1, k);
            }
        }
    }
    int bx[6] = {BOX_EMPTY, BOX_EMPTY, BOX_EMPTY, BOX_EMPTY, BOX_EMPTY, BOX_EMPTY};
    if (ilo != BOX_EMPTY) {       // in the frame: (i, j) or, swapped, (j, i)
        bx[0] = swp ? j : ilo; bx[1] = swp ? ilo : j; bx[2] = k;
        bx[3] = swp ? -j : ihi; bx[4] = swp ? ihi : -j; bx[5] = -k;
    }
    box_reduce(bx, box_out);      // every thread of the block, one call site
}

inline bool aligned(const void* p, unsigned a) { return p == nullptr || ((uintptr_t)p & (a - 1)) == 0; }

inline unsigned blocks_for(long work) { return (unsigned)((work + kWarpThreads - 1) / kWarpThreads); }

// Launch shape of the solver warps (see k_warp_pca): per = voxels along x per
// thread; threads per block = the row's threads rounded up to a warp, at most
// kWarpThreads.
struct RowLaunch {
    dim3 grid;
    unsigned threads;
};
inline RowLaunch row_launch(const Grid& g, int per) {
    const int need = (g.nx + per - 1) / per;
    const int t = need >= kWarpThreads ? kWarpThreads : ((need + 31) / 32) * 32;
    return {dim3((unsigned)((need + t - 1) / t), (unsigned)g.ny, (unsigned)g.nz), (unsigned)t};
}

template <typename T>
cudaError_t pca_dvf_t(const void* mean, const void* U, int K, const float* w, Grid g, float* dvf,
                      cudaStream_t s) {
    long N = (long)g.nx * g.ny * g.nz;
    WSrc ws{};
    for (int k = 0; k < K && k < PCAS_KMAX; k++) ws.w[k] = w[k];
    const unsigned a = sizeof(T) * 4;
    bool vec = (N % 4 == 0) && aligned(mean, a) && aligned(U, a) && aligned(dvf, 16);
    const T* m = static_cast<const T*>(mean);
    const T* u = static_cast<const T*>(U);
    if (vec) k_pca_dvf<true, T><<<blocks_for(N / 4), kWarpThreads, 0, s>>>(m, u, K, ws, N, dvf);
    else k_pca_dvf<false, T><<<blocks_for(N), kWarpThreads, 0, s>>>(m, u, K, ws, N, dvf);
    return cudaGetLastError();
}

template <typename T>
cudaError_t warp_pca_t(const float* f, const void* mean, const void* U, int K, WSrc w, Grid g,
                       const View* Vd, float* fpad, float2* fpair, int* box, Occ oc, cudaStream_t s) {
    const unsigned a = sizeof(T) * 4;
    bool vec = (g.nx % 4 == 0) && aligned(mean, a) && aligned(U, a) && aligned(fpad, 16) && aligned(fpair, 16);
    const T* m = static_cast<const T*>(mean);
    const T* u = static_cast<const T*>(U);
    const RowLaunch L = row_launch(g, vec ? 4 : 1);
    if (vec) k_warp_pca<true, T><<<L.grid, L.threads, 0, s>>>(f, m, u, K, w, g, Vd, fpad, fpair, box, oc);
    else k_warp_pca<false, T><<<L.grid, L.threads, 0, s>>>(f, m, u, K, w, g, Vd, fpad, fpair, box, oc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t warp_batch_t(const float* f0, const T* mean, const T* U, int K, const SolveState* st, Grid g,
                         const View* Vd, float4* fpad4, float* fpad, int* box, Occ oc, const RowLaunch& L,
                         cudaStream_t s) {
    switch (K) {
#define PCAS_WB_CASE(KK) \
        case KK: k_warp_batch<T, KK, kBatchVPT><<<L.grid, L.threads, 0, s>>>(f0, mean, U, st, g, Vd, fpad4, fpad, box, oc); break;
        PCAS_WB_CASE(1) PCAS_WB_CASE(2) PCAS_WB_CASE(3) PCAS_WB_CASE(4)
        PCAS_WB_CASE(5) PCAS_WB_CASE(6) PCAS_WB_CASE(7) PCAS_WB_CASE(8)
#undef PCAS_WB_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

#define PCAS_DT_DISPATCH(dt, CALL)                                         \
    switch (dt) {                                                          \
        case DT_F32: { using T = float; return CALL; }                     \
        case DT_BF16: { using T = __nv_bfloat16; return CALL; }            \
        case DT_F16: { using T = __half; return CALL; }                    \
        default: return cudaErrorInvalidValue;                             \
    }

cudaError_t launch_pca_dvf(const void* mean, const void* U, int dt, int K, const float* w, Grid g,
                           float* dvf, cudaStream_t s) {
    PCAS_DT_DISPATCH(dt, (pca_dvf_t<T>(mean, U, K, w, g, dvf, s)))
}

cudaError_t launch_warp_dvf(const void* f0, int dt, const float* dvf, Grid g, float* f, cudaStream_t s) {
    long N = (long)g.nx * g.ny * g.nz;
    PCAS_DT_DISPATCH(dt, (k_warp_dvf<T><<<blocks_for(N), kWarpThreads, 0, s>>>(static_cast<const T*>(f0), dvf, g,
                                                                              N, f),
                          cudaGetLastError()))
}

cudaError_t launch_fill_f0h(const void* f0, int dt, Grid g, float* f0h, unsigned char* f0m, const int* skip,
                            cudaStream_t s) {
    const int rows = g.ny * g.nz;
    const unsigned nb = (unsigned)(rows < 1216 ? rows : 1216);     // 8 blocks per SM of a GB300
    PCAS_DT_DISPATCH(dt, (k_fill_f0h<T><<<nb, kWarpThreads, 0, s>>>(static_cast<const T*>(f0), g, f0h, f0m, skip),
                          cudaGetLastError()))
}

cudaError_t launch_warp_pca(const float* f0, const void* mean, const void* U, int dt, int K, WSrc w,
                            Grid g, const View* Vd, float* fpad, float2* fpair, int* box, Occ oc, cudaStream_t s) {
    PCAS_DT_DISPATCH(dt, (warp_pca_t<T>(f0, mean, U, K, w, g, Vd, fpad, fpair, box, oc, s)))
}

cudaError_t launch_warp_batch(const float* f0, const void* mean, const void* U, int dt, int K,
                              const SolveState* st, Grid g, const View* Vd, float4* fpad4, float* fpad,
                              Occ oc, cudaStream_t s) {
    const RowLaunch L = row_launch(g, kBatchVPT);
    int* box = const_cast<int*>(st->box[1]);
    PCAS_DT_DISPATCH(dt, (warp_batch_t<T>(f0, static_cast<const T*>(mean),
                                          static_cast<const T*>(U), K, st, g, Vd, fpad4, fpad, box, oc, L, s)))
}

#undef PCAS_DT_DISPATCH

}  // namespace pcas
