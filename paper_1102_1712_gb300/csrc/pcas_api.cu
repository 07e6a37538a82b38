// pcas_api.cu -- the C ABI of libpcasolve (declared in include/pcasolve.h):
// argument checks, view geometry in FP64 on the host, workspace layout, the
// solve loop of the Appendix, and the small kernels (state set-up, tumour
// localisation of Sec. II.A).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <vector>

#include "pcas_internal.cuh"

using namespace pcas;

__device__ double d_localize_out[4];

namespace {

thread_local char g_err[512] = "";
std::mutex g_localize_mutex;

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define PCAS_CUDA(call)                                                                \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(PCAS_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)


// ------------------------------------------------------------- profiling
// Launch counts per kernel class (always) and, while enabled, CUDA-event
// brackets around each launch, recorded on the launch stream.
constexpr int kProfSlots = 65536;
std::mutex g_prof_mutex;
long long g_launches[PCAS_K_COUNT];
bool g_prof_on = false;
cudaEvent_t* g_ev = nullptr;           // 2 * kProfSlots events, created once
int g_ev_kind[kProfSlots];
int g_ev_used = 0;

// Per-thread event timing used by the autotuner (independent of the global
// profiler; the autotuner's launches are not counted there).
constexpr int kLocalSlots = 8192;
constexpr int kLocalBase = 1 << 24;
struct LocalTimer {
    cudaEvent_t ev[2 * kLocalSlots];
    int kind[kLocalSlots];
    int used = 0;
    int created = 0;           // events created so far (lazily)
};
thread_local LocalTimer* t_local = nullptr;

int prof_begin(int kind, cudaStream_t s) {
    if (t_local) {
        LocalTimer& L = *t_local;
        if (L.used >= kLocalSlots) return -1;
        const int slot = L.used++;
        if (2 * slot + 1 >= L.created) {
            if (cudaEventCreate(&L.ev[2 * slot]) != cudaSuccess) return -1;
            if (cudaEventCreate(&L.ev[2 * slot + 1]) != cudaSuccess) return -1;
            L.created = 2 * slot + 2;
        }
        L.kind[slot] = kind;
        cudaEventRecord(L.ev[2 * slot], s);
        return kLocalBase + slot;
    }
    std::lock_guard<std::mutex> lk(g_prof_mutex);
    g_launches[kind]++;
    if (!g_prof_on || !g_ev || g_ev_used >= kProfSlots) return -1;
    int slot = g_ev_used++;
    g_ev_kind[slot] = kind;
    cudaEventRecord(g_ev[2 * slot], s);
    return slot;
}

void prof_end(int slot, cudaStream_t s) {
    if (slot < 0) return;
    if (slot >= kLocalBase) {
        cudaEventRecord(t_local->ev[2 * (slot - kLocalBase) + 1], s);
        return;
    }
    cudaEventRecord(g_ev[2 * slot + 1], s);
}

#define PCAS_LAUNCH(kind, s, expr)                                                          \
    do {                                                                                    \
        int slot_ = prof_begin((kind), (s));                                                \
        cudaError_t e_ = (expr);                                                            \
        prof_end(slot_, (s));                                                               \
        if (e_ != cudaSuccess)                                                              \
            return fail(PCAS_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));     \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

int check_vol(const pcas_vol* v) {
    if (!v) return fail(PCAS_ERR_INVALID_ARG, "vol is NULL");
    if (v->nx < 1 || v->ny < 1 || v->nz < 1)
        return fail(PCAS_ERR_INVALID_ARG, "volume dims must be positive (%d,%d,%d)", v->nx, v->ny, v->nz);
    // 32-bit voxel offsets: either zero-halo layout of the warped volume (at
    // most (m + 10) (m + 4) (nz + 4) elements, m = max(nx, ny)) and the
    // reference CT's halo copy ((nx + 6) (ny + 6) (nz + 6) elements) stay below
    // 2^31; ny, nz index grid rows
    const double m = v->nx > v->ny ? v->nx : v->ny;
    if ((m + 10.0) * (m + 4.0) * (v->nz + 4.0) > 2147483647.0 ||
        (v->nx + 6.0) * (v->ny + 6.0) * (v->nz + 6.0) > 2147483647.0 || v->ny > 65535 || v->nz > 65535)
        return fail(PCAS_ERR_INVALID_ARG, "volume too large (%d,%d,%d): at most 2^31 voxels with halo, "
                    "ny and nz at most 65535", v->nx, v->ny, v->nz);
    if (!(v->sx > 0) || !(v->sy > 0) || !(v->sz > 0))
        return fail(PCAS_ERR_INVALID_ARG, "voxel spacing must be positive");
    if (!isfinite(v->ox) || !isfinite(v->oy) || !isfinite(v->oz))
        return fail(PCAS_ERR_INVALID_ARG, "volume origin must be finite");
    return PCAS_OK;
}

Grid make_grid(const pcas_vol* v) {
    Grid g;
    g.nx = v->nx; g.ny = v->ny; g.nz = v->nz;
    g.inv_sx = (float)(1.0 / v->sx); g.inv_sy = (float)(1.0 / v->sy); g.inv_sz = (float)(1.0 / v->sz);
    return g;
}

// View geometry (header comment of pcasolve.h) in FP64, then rounded once.
int make_view(const pcas_vol* vol, const pcas_cb* cb, double step, View* V) {
    if (!cb) return fail(PCAS_ERR_INVALID_ARG, "cb is NULL");
    if (cb->nu < 1 || cb->nv < 1 || (double)cb->nu * cb->nv > 1.0e9)
        return fail(PCAS_ERR_INVALID_ARG, "detector size invalid (%d x %d)", cb->nu, cb->nv);
    if (!(cb->sad > 0) || !(cb->sdd > 0) || !(cb->du > 0) || !(cb->dv > 0) || !isfinite(cb->angle_rad) ||
        !isfinite(cb->off_u) || !isfinite(cb->off_v) || !isfinite(cb->sad) || !isfinite(cb->sdd))
        return fail(PCAS_ERR_INVALID_ARG, "cone-beam geometry invalid");
    if (!(step > 0) || !isfinite(step)) return fail(PCAS_ERR_INVALID_ARG, "step_mm must be > 0");
    const double sa = sin(cb->angle_rad), ca = cos(cb->angle_rad);
    const double S[3] = {cb->sad * sa, -cb->sad * ca, 0.0};
    const double ew[3] = {-sa, ca, 0.0}, eu[3] = {ca, sa, 0.0}, ev[3] = {0.0, 0.0, 1.0};
    const double o[3] = {vol->ox, vol->oy, vol->oz}, s[3] = {vol->sx, vol->sy, vol->sz};
    const int n[3] = {vol->nx, vol->ny, vol->nz};
    for (int corner = 0; corner < 8; corner++) {   // whole support box ahead of the source
        double dot = 0;
        for (int c = 0; c < 3; c++) {
            double X = (corner >> c & 1) ? o[c] + n[c] * s[c] : o[c] - s[c];
            dot += (X - S[c]) * ew[c];
        }
        if (!(dot > 0))
            return fail(PCAS_ERR_INVALID_ARG, "the volume must lie entirely in front of the source");
    }
    if ((double)cb->sdd * 4.0 > 1e30) return fail(PCAS_ERR_INVALID_ARG, "sdd too large");
    // sample indices i = t/step must stay far inside the int range
    double far = cb->sad + 2.0 * (n[0] * s[0] + n[1] * s[1] + n[2] * s[2]);
    if (far / step > 1.0e8) return fail(PCAS_ERR_INVALID_ARG, "step_mm too small for this geometry");
    V->Q0 = make_float3((float)((S[0] - o[0]) / s[0]), (float)((S[1] - o[1]) / s[1]),
                        (float)((S[2] - o[2]) / s[2]));
    V->A = make_float3((float)(cb->sdd * ew[0] / s[0]), (float)(cb->sdd * ew[1] / s[1]),
                       (float)(cb->sdd * ew[2] / s[2]));
    V->Bu = make_float3((float)(eu[0] / s[0]), (float)(eu[1] / s[1]), (float)(eu[2] / s[2]));
    V->Bv = make_float3((float)(ev[0] / s[0]), (float)(ev[1] / s[1]), (float)(ev[2] / s[2]));
    V->EW = make_float3((float)(ew[0] * s[0]), (float)(ew[1] * s[1]), (float)(ew[2] * s[2]));
    V->EU = make_float3((float)(eu[0] * s[0]), (float)(eu[1] * s[1]), (float)(eu[2] * s[2]));
    V->EV = make_float3((float)(ev[0] * s[0]), (float)(ev[1] * s[1]), (float)(ev[2] * s[2]));
    V->sdd = (float)cb->sdd;
    V->sdd2 = (float)(cb->sdd * cb->sdd);
    V->u0 = (float)(cb->off_u - 0.5 * (cb->nu - 1) * cb->du);
    V->v0 = (float)(cb->off_v - 0.5 * (cb->nv - 1) * cb->dv);
    V->du = (float)cb->du;
    V->dv = (float)cb->dv;
    V->nu = cb->nu;
    V->nv = cb->nv;
    V->step = (float)step;
    V->swap = 0;                            // launch shapes: set_layouts
    V->lw1 = V->lw4 = 3;
    V->chunk1 = 0;
    V->chunk4 = 16;
    V->pt_rect = nullptr;                   // no fixed-view cache: pcas_solver_fix_view
    V->pt_off = nullptr;
    V->pt_w = nullptr;
    return PCAS_OK;
}

int check_model(const void* mean, const void* U, int K) {
    (void)mean;
    if (K < 1 || K > PCAS_KMAX) return fail(PCAS_ERR_INVALID_ARG, "K must be in [1, %d], got %d", PCAS_KMAX, K);
    if (!U) return fail(PCAS_ERR_INVALID_ARG, "U is NULL");
    return PCAS_OK;
}

// ------------------------------------------------------------- workspace
struct Layout {
    size_t state, view, f0h, f0m, fpad, fpair, fpad4, occ, pbuf, rayt, part_drr, part_res, part_adj, act_idx, act_h,
        tile_count, tile_off, total;
};

Layout layout(const pcas_vol* vol, const pcas_cb* cb, int K) {
    Layout L;
    // room for either solver layout (x fastest or y fastest)
    const Pad pa = solver_pad(vol->nx, vol->ny, vol->nz, 0), pb = solver_pad(vol->nx, vol->ny, vol->nz, 1);
    const size_t na = (size_t)pa.px * pa.pny * pa.pnz, nb = (size_t)pb.px * pb.pny * pb.pnz;
    const size_t npad = na > nb ? na : nb;
    size_t M = (size_t)cb->nu * cb->nv;
    size_t off = 0;
    L.state = off; off += align256(sizeof(SolveState));
    L.view = off; off += align256(sizeof(View));
    L.f0h = off; off += align256((size_t)f0h_count(vol->nx, vol->ny, vol->nz) * sizeof(float));  // f0, halo 3
    L.f0m = off; off += align256((size_t)f0b_count(vol->nx, vol->ny, vol->nz));     // its bricks (zeroed with it)
    L.fpad = off; off += align256(npad * sizeof(float));                 // f(w), zero halo
    L.fpair = off; off += align256(npad * sizeof(float2));               // f(w) as x pairs (the L1 march)
    L.fpad4 = off; off += align256(npad * sizeof(float4));               // candidates 0-3 (4 in fpad)
    L.occ = off; off += align256((size_t)occ_count(vol->nx, vol->ny, vol->nz) * sizeof(unsigned int));
    L.pbuf = off; off += align256((size_t)NBUF * M * sizeof(float));     // projection ring
    L.rayt = off; off += align256(2 * M * sizeof(float4) + M * sizeof(float));   // (step, r), (1/step, 0); r
    L.part_drr = off; off += align256((size_t)drr_blocks(cb->nu, cb->nv) * DRR_PART_VALS * sizeof(double));
    L.part_res = off; off += align256((size_t)resid_blocks(cb->nu, cb->nv) * sizeof(double));
    L.part_adj = off; off += align256((size_t)ADJ_MAX_BLOCKS * PCAS_KMAX * sizeof(double));
    const size_t nt = (size_t)adj_tiles_max(vol->nx, vol->ny, vol->nz), cap = nt * 256;
    L.act_idx = off; off += align256(cap * sizeof(int));                  // compacted voxels
    L.act_h = off; off += align256((size_t)K * cap * sizeof(float));
    L.tile_count = off; off += align256(nt * sizeof(int));
    L.tile_off = off; off += align256((nt + 1) * sizeof(int));
    L.total = off;
    return L;
}

struct Ws {
    SolveState* st;
    View* view;
    float* f0h;
    unsigned char* f0m;       // bricks of the reference CT, right after f0h
    size_t f0h_bytes;         // f0h and f0m
    unsigned int* occ;        // occupancy bricks of the solver volumes
    float *fpad, *pbuf;
    float2* fpair;
    float4 *fpad4, *rayt;
    double *part_drr, *part_res, *part_adj;
    size_t fpad_bytes, fpad4_bytes;      // fpad_bytes: fpad and fpair
    AdjScratch adj;
};

int bind_ws(void* ws, size_t ws_bytes, const pcas_vol* vol, const pcas_cb* cb, int K, Ws* W) {
    Layout L = layout(vol, cb, K);
    if (!ws) return fail(PCAS_ERR_INVALID_ARG, "workspace is NULL");
    if (((uintptr_t)ws & 255u) != 0) return fail(PCAS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < L.total)
        return fail(PCAS_ERR_INVALID_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, L.total);
    char* b = static_cast<char*>(ws);
    W->st = reinterpret_cast<SolveState*>(b + L.state);
    W->view = reinterpret_cast<View*>(b + L.view);
    W->f0h = reinterpret_cast<float*>(b + L.f0h);
    W->f0m = reinterpret_cast<unsigned char*>(b + L.f0m);
    W->f0h_bytes = L.fpad - L.f0h;
    W->fpad = reinterpret_cast<float*>(b + L.fpad);
    W->fpair = reinterpret_cast<float2*>(b + L.fpair);
    W->fpad4 = reinterpret_cast<float4*>(b + L.fpad4);
    W->occ = reinterpret_cast<unsigned int*>(b + L.occ);
    W->pbuf = reinterpret_cast<float*>(b + L.pbuf);
    W->rayt = reinterpret_cast<float4*>(b + L.rayt);
    W->part_drr = reinterpret_cast<double*>(b + L.part_drr);
    W->part_res = reinterpret_cast<double*>(b + L.part_res);
    W->part_adj = reinterpret_cast<double*>(b + L.part_adj);
    W->adj.act_idx = reinterpret_cast<int*>(b + L.act_idx);
    W->adj.act_h = reinterpret_cast<float*>(b + L.act_h);
    W->adj.tile_count = reinterpret_cast<int*>(b + L.tile_count);
    W->adj.tile_off = reinterpret_cast<int*>(b + L.tile_off);
    W->fpad_bytes = L.fpad4 - L.fpad;
    W->fpad4_bytes = L.occ - L.fpad4;
    return PCAS_OK;
}

// Occupancy bricks as the solver kernels take them (skipping off: none).
inline Occ occ_of(const Ws& W, const Tune& T) {
    return Occ{T.skip ? W.occ : nullptr, &W.st->occ_gen, T.skip ? W.f0m : nullptr};
}

// Where the one-volume warp writes f(w): its x-pair copy, which the one-volume
// projector reads (through L1, or staged chunk by chunk).
inline float2* pair_of(const Ws& W, const Tune&) { return W.fpair; }

// The first evaluation's warp of a solve at the staged w (st->w), fused with
// the Jacobian pass of the gradient at that w (launch_warp_jac): the next
// launch_adjoint_grad with T.vt skips its own.
inline cudaError_t first_warp(const Ws& W, const Tune& T, const Grid& g, const void* mean, const void* U, int dt,
                              int K, cudaStream_t s) {
    const Occ oc = occ_of(W, T);
    const JacWarp jw{W.view, W.fpad, pair_of(W, T), W.st->box[0], oc};
    return launch_warp_jac(g, W.f0h, oc.f0m, mean, U, dt, K, W.st, W.adj, T.vt, jw, s);
}

// ------------------------------------------------------------ launch shapes
// Default shapes: 8 x 4 warp patches, 16-sample chunks for the batch
// projector (the one-volume projector marches through L1), 8 x 8 x 4 voxel tiles,
// eight gather blocks per SM, empty-space skipping on, y-fastest solver
// volumes for angles near 90 (bins 67.5 ... 112.5 degrees).
Tune default_tune() {
    Tune T;
    T.lw1 = 3;
    T.chunk1 = 0;
    T.vt = 0;
    T.adj_mult = 8;
    T.skip = 1;
    for (int b = 0; b < NBIN; b++) {
        T.lw4[b] = 3;
        T.chunk4[b] = 16;
        T.swap[b] = (b >= 3 && b <= 5) ? 1 : 0;
    }
    return T;
}

// 22.5-degree bin of the gantry angle modulo 180 degrees, bins centred on
// 0, 22.5, ..., 157.5 degrees.
int angle_bin(double angle) {
    double a = fmod(angle, M_PI);
    if (a < 0) a += M_PI;
    int b = (int)floor(a / (M_PI / NBIN) + 0.5);
    return b % NBIN;
}

void set_layouts(View& V, const Tune& T, double angle) {
    const int b = angle_bin(angle);
    V.swap = T.swap[b];
    V.lw1 = T.lw1;
    V.lw4 = T.lw4[b];
    V.chunk1 = T.chunk1;
    V.chunk4 = T.chunk4[b];
}

// Size buckets: volume extents in steps of 32 (x, y) and 16 (z) voxels,
// detector extents in steps of 64 pixels, K and the storage type.
struct BucketKey {
    int bx, by, bz, bu, bv, K, dt;
    bool operator<(const BucketKey& o) const {
        const int a[7] = {bx, by, bz, bu, bv, K, dt}, c[7] = {o.bx, o.by, o.bz, o.bu, o.bv, o.K, o.dt};
        for (int i = 0; i < 7; i++)
            if (a[i] != c[i]) return a[i] < c[i];
        return false;
    }
};
BucketKey bucket_of(const pcas_vol* vol, const pcas_cb* cb, int K, int dt) {
    return {(vol->nx + 31) / 32, (vol->ny + 31) / 32, (vol->nz + 15) / 16, (cb->nu + 63) / 64, (cb->nv + 63) / 64,
            K, dt};
}
std::mutex g_tune_mutex;
std::map<BucketKey, Tune> g_tunes;

Tune tune_for(const pcas_vol* vol, const pcas_cb* cb, int K, int dt) {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    auto it = g_tunes.find(bucket_of(vol, cb, K, dt));
    return it == g_tunes.end() ? default_tune() : it->second;
}

int gather_blocks(const Tune& T) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        sms = 152;
    const int nb = T.adj_mult * sms;
    return nb < 1 ? 1 : (nb > ADJ_MAX_BLOCKS ? ADJ_MAX_BLOCKS : nb);
}

// ------------------------------------------------------------ small kernels
// Sum over lanes 0..7 (the other lanes hold zeros), returned to every lane:
// the value of a sum over the warp, without its two levels that add zeros.
__device__ __forceinline__ double tap_sum8(double v) {
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return __shfl_sync(0xffffffffu, v, 0);
}

// Sec. II.A fixed point c = c_ref - x(c) for the tumour centroid, by one warp:
// lanes 0..7 own the eight taps of the trilinear DVF sample (Eq. 1 at w), each
// loading its tap's model values only when the iterate moves to another cell.
// Lane 0 writes out[0..2] = c and out[3] = 1 if it converged (else 0).
template <typename T>
__device__ void localize_warp(const T* __restrict__ mean, const T* __restrict__ U, int K, const Grid& g,
                              const double* w, double ox, double oy, double oz, double isx, double isy,
                              double isz, double cx, double cy, double cz, int max_iter, double tol,
                              double* out) {
    const int lane = threadIdx.x;
    const long N = (long)g.nx * g.ny * g.nz;
    double y[3] = {0.0, 0.0, 0.0};
    int converged = 0, it = 0;
    // mean + U w at this lane's tap voxel, kept while the iterates stay in one
    // cell (the same values, computed once instead of once per iteration)
    long vhold = -1;
    double xv[3] = {0.0, 0.0, 0.0};
    for (; it < max_iter; it++) {
        double q[3] = {(cx + y[0] - ox) * isx, (cy + y[1] - oy) * isy, (cz + y[2] - oz) * isz};
        double x[3] = {0.0, 0.0, 0.0};
        if (lane < 8) {
            bool inside = true;
            double f[3];
            long idx[3];
            const int n[3] = {g.nx, g.ny, g.nz};
            for (int c = 0; c < 3; c++) {
                double qc = fmin(fmax(q[c], -2.0), (double)n[c] + 1.0);
                double fl = floor(qc);
                int bit = (lane >> c) & 1;
                double z = qc - fl;
                long l = (long)fl + bit;
                f[c] = bit ? z : 1.0 - z;
                inside = inside && l >= 0 && l < n[c];
                idx[c] = l;
            }
            const double wt = (f[0] * f[1]) * f[2];
            if (inside && wt != 0.0) {
                long v = (idx[2] * g.ny + idx[1]) * g.nx + idx[0];
                if (v != vhold) {
                    for (int c = 0; c < 3; c++) {
                        double val = mean ? (double)ldg_f(mean + c * N + v) : 0.0;
                        for (int k = 0; k < K; k++) val += w[k] * (double)ldg_f(U + ((long)k * 3 + c) * N + v);
                        xv[c] = val;
                    }
                    vhold = v;
                }
                for (int c = 0; c < 3; c++) x[c] = wt * xv[c];
            }
        }
        double change = 0.0;
        for (int c = 0; c < 3; c++) {
            double s = tap_sum8(x[c]);
            double yn = -s;
            change = fmax(change, fabs(yn - y[c]));
            y[c] = yn;
        }
        if (change < tol) { converged = 1; break; }
    }
    if (lane == 0) {
        out[0] = cx + y[0];
        out[1] = cy + y[1];
        out[2] = cz + y[2];
        out[3] = converged ? 1.0 : 0.0;
    }
}

template <typename T>
__global__ void k_localize(const T* __restrict__ mean, const T* __restrict__ U, int K,
                           Grid g, double w0, double w1, double w2, double w3, double w4, double w5,
                           double w6, double w7, double ox, double oy, double oz, double isx,
                           double isy, double isz, double cx, double cy, double cz, int max_iter,
                           double tol, double* out) {
    const double w[PCAS_KMAX] = {w0, w1, w2, w3, w4, w5, w6, w7};
    localize_warp(mean, U, K, g, w, ox, oy, oz, isx, isy, isz, cx, cy, cz, max_iter, tol, out);
}

// Reset the solver state for a new evaluation/solve.
__global__ void k_init_state(SolveState* st, int K, double w0, double w1, double w2, double w3,
                             double w4, double w5, double w6, double w7, double mu0, double alpha,
                             double beta, double mu_min, int max_trials, int max_iter) {
    if (threadIdx.x != 0) return;
    const double w[PCAS_KMAX] = {w0, w1, w2, w3, w4, w5, w6, w7};
    for (int k = 0; k < PCAS_KMAX; k++) {
        st->w[k] = k < K ? w[k] : 0.0;
        st->d[k] = 0.0;
        st->G[k] = 0.0;
        for (int j = 0; j < TRIAL_BATCH; j++) st->wt[j][k] = st->w[k];
    }
    for (int j = 0; j < TRIAL_BATCH; j++) st->mu_batch[j] = 0.0;
    st->gnorm = st->a = st->b = st->J = st->J0 = st->Jt = 0.0;
    st->mu = mu0;
    for (int i = 0; i < NBUF; i++)
        for (int j = 0; j < NMOM; j++) st->mom[i][j] = 0.0;
    st->mu0 = mu0; st->alpha = alpha; st->beta = beta; st->mu_min = mu_min;
    st->K = K; st->max_trials = max_trials;
    st->cur = 0; st->phase = PH_RUNNING; st->evals = 0; st->trials = 0;
    st->nvalid = 0; st->iters = 0; st->batches = 0; st->max_iter = max_iter; st->launches = 0;
    st->wide = 1;
    st->jac_ready = 0;
    for (int i = 0; i < 4; i++) st->counter[i] = 0u;
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 6; j++) st->box[i][j] = BOX_EMPTY;
}

int upload_view(View* dst, const View& V, cudaStream_t s) {
    PCAS_CUDA(cudaMemcpyAsync(dst, &V, sizeof(View), cudaMemcpyHostToDevice, s));
    return PCAS_OK;
}

int launch_init(SolveState* st, int K, const double* w, const pcas_params* prm, cudaStream_t s) {
    double v[PCAS_KMAX] = {0};
    for (int k = 0; k < K; k++) v[k] = w[k];
    pcas_params d = {0.2, 0.1, 0.5, 0.01, 10, 30, 1.0};
    if (!prm) prm = &d;
    PCAS_LAUNCH(PCAS_K_INIT, s,
                (k_init_state<<<1, 32, 0, s>>>(st, K, v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7],
                                               prm->mu0, prm->alpha, prm->beta, prm->mu_min,
                                               prm->max_trials, prm->max_iter),
                 cudaGetLastError()));
    return PCAS_OK;
}

int check_dtype(int dt) {
    if (dt != PCAS_F32 && dt != PCAS_BF16 && dt != PCAS_F16)
        return fail(PCAS_ERR_INVALID_ARG, "storage dtype must be PCAS_F32, PCAS_BF16 or PCAS_F16, got %d", dt);
    return PCAS_OK;
}

int check_ptr(const void* p, const char* name) {
    if (!p) return fail(PCAS_ERR_INVALID_ARG, "%s is NULL", name);
    return PCAS_OK;
}

int check_finite(const double* v, int n, const char* name) {
    for (int i = 0; i < n; i++)
        if (!isfinite(v[i])) return fail(PCAS_ERR_INVALID_ARG, "%s[%d] is not finite", name, i);
    return PCAS_OK;
}

#define PCAS_TRY(x)              \
    do {                         \
        int rc_ = (x);           \
        if (rc_ != PCAS_OK) return rc_; \
    } while (0)

// The halo copy of the reference CT for this call and its bricks (zeroed,
// then filled).
int stage_f0h(const void* f0, int dt, const Grid& g, const Ws& W, const Tune& T, cudaStream_t s) {
    PCAS_CUDA(cudaMemsetAsync(W.f0h, 0, W.f0h_bytes, s));
    PCAS_LAUNCH(PCAS_K_INIT, s, launch_fill_f0h(f0, dt, g, W.f0h, T.skip ? W.f0m : nullptr, nullptr, s));
    return PCAS_OK;
}

// Everything up to and including the gradient at st->w: warp, DRR with
// moments, (A.1) + residual + J, fused adjoint gradient.
int eval_gradient_pipeline(const void* f0, const void* mean, const void* U, int dt, int K, const float* y,
                           const Grid& g, const View& V, const Ws& W, int step_setup, const Tune& T,
                           cudaStream_t s) {
    PCAS_TRY(stage_f0h(f0, dt, g, W, T, s));
    PCAS_LAUNCH(PCAS_K_WARP_PCA, s, first_warp(W, T, g, mean, U, dt, K, s));
    PCAS_LAUNCH(PCAS_K_DRR_SOLVER, s,
                launch_drr_solver(W.fpad, W.fpair, W.fpad4, g, V, W.view, y, W.pbuf, 0, W.st, W.part_drr, T, 0ull, 0,
                                  occ_of(W, T), s));
    PCAS_LAUNCH(PCAS_K_RESID, s, launch_resid(W.pbuf, y, V, W.view, 1, W.rayt, W.st, W.part_res, s));
    PCAS_LAUNCH(PCAS_K_ADJ_GRAD, s,
                launch_adjoint_grad(W.rayt, g, W.view, W.f0h, occ_of(W, T).f0m, mean, U, dt, K, step_setup, W.st,
                                    W.part_adj, W.adj, T.vt, gather_blocks(T), 0ull, 0, nullptr, s));
    return PCAS_OK;
}

// The host-driven solve (solve_projection) with launch shapes T.
int solve_host(const void* f0, const void* mean, const void* U, int dtype, int K, const float* y,
               const pcas_vol* vol, const pcas_cb* cb, const double* w_init, const pcas_params* prm,
               const Tune& T, double* w_out, pcas_stats* stats, void* ws, size_t ws_bytes, cudaStream_t s) {
    View V;
    PCAS_TRY(make_view(vol, cb, prm->step_mm, &V));
    set_layouts(V, T, cb->angle_rad);
    Ws W;
    PCAS_TRY(bind_ws(ws, ws_bytes, vol, cb, K, &W));
    Grid g = make_grid(vol);
    const int adj_blocks = gather_blocks(T);
    PCAS_CUDA(cudaMemsetAsync(W.fpad, 0, W.fpad_bytes + W.fpad4_bytes, s));   // zero halos
    PCAS_TRY(launch_init(W.st, K, w_init, prm, s));
    PCAS_TRY(upload_view(W.view, V, s));
    PCAS_TRY(stage_f0h(f0, dtype, g, W, T, s));
    PCAS_LAUNCH(PCAS_K_WARP_PCA, s, first_warp(W, T, g, mean, U, dtype, K, s));
    PCAS_LAUNCH(PCAS_K_DRR_SOLVER, s,
                launch_drr_solver(W.fpad, W.fpair, W.fpad4, g, V, W.view, y, W.pbuf, 0, W.st, W.part_drr, T, 0ull, 0,
                                  occ_of(W, T), s));
    int iters = 0, phase = PH_RUNNING;
    for (int it = 0; it < prm->max_iter; it++) {
        PCAS_LAUNCH(PCAS_K_RESID, s, launch_resid(W.pbuf, y, V, W.view, it == 0, W.rayt, W.st, W.part_res, s));
        PCAS_LAUNCH(PCAS_K_ADJ_GRAD, s,
                    launch_adjoint_grad(W.rayt, g, W.view, W.f0h, occ_of(W, T).f0m, mean, U, dtype, K, 1, W.st,
                                        W.part_adj, W.adj, T.vt, adj_blocks, 0ull, 0, nullptr, s));
        // Armijo backtracking over the schedule mu0, beta mu0, ...: the next
        // step sizes that the rule may still try (up to five, two after an
        // iteration that took its first one) are rendered and tested in one
        // pass; the device accepts the first that passes, in order, and stops
        // when the schedule is spent.  The host reads one flag per batch.
        phase = PH_RUNNING;
        for (int batch = 0; batch <= prm->max_trials; batch++) {    // each batch tries >= 1 step
            PCAS_LAUNCH(PCAS_K_WARP_BATCH, s, launch_warp_batch(W.f0h, mean, U, dtype, K, W.st, g, W.view,
                                                                W.fpad4, W.fpad, occ_of(W, T), s));
            PCAS_LAUNCH(PCAS_K_DRR_BATCH, s,
                        launch_drr_solver(W.fpad, W.fpair, W.fpad4, g, V, W.view, y, W.pbuf, TRIAL_BATCH, W.st, W.part_drr,
                                          T, 0ull, 0, occ_of(W, T), s));
            PCAS_CUDA(cudaMemcpyAsync(&phase, &W.st->phase, sizeof(int), cudaMemcpyDeviceToHost, s));
            PCAS_CUDA(cudaStreamSynchronize(s));
            if (phase != PH_RUNNING) break;
        }
        if (phase == PH_RUNNING) phase = PH_STOP;     // batch cap reached without a decision
        if (phase == PH_ACCEPT || phase == PH_STOP) iters++;
        if (phase != PH_ACCEPT) break;
    }
    SolveState h;
    PCAS_CUDA(cudaMemcpyAsync(&h, W.st, sizeof(h), cudaMemcpyDeviceToHost, s));
    PCAS_CUDA(cudaStreamSynchronize(s));
    if (h.phase == PH_SINGULAR) return fail(PCAS_ERR_SINGULAR, "Y^T Y is singular (constant image y)");
    for (int k = 0; k < K; k++) w_out[k] = h.w[k];
    if (stats) {
        stats->iters = iters;
        stats->evals = h.evals;
        stats->status = PCAS_OK;
        stats->J0 = h.J0;
        stats->J = h.J;
        stats->a = h.a;
        stats->b = h.b;
        stats->mu_last = h.mu;
    }
    return PCAS_OK;
}

}  // namespace

extern "C" {

int pcas_profile(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mutex);
    for (int k = 0; k < PCAS_K_COUNT; k++) g_launches[k] = 0;
    g_ev_used = 0;
    if (on && !g_ev) {
        cudaEvent_t* ev = new cudaEvent_t[2 * kProfSlots];
        for (int i = 0; i < 2 * kProfSlots; i++) {
            cudaError_t e = cudaEventCreate(&ev[i]);
            if (e != cudaSuccess) {
                for (int j = 0; j < i; j++) cudaEventDestroy(ev[j]);
                delete[] ev;
                return fail(PCAS_ERR_CUDA, "cudaEventCreate failed: %s", cudaGetErrorString(e));
            }
        }
        g_ev = ev;
    }
    g_prof_on = on != 0;
    return PCAS_OK;
}

int pcas_profile_read(int kind, long long* launches, double* total_ms) {
    if (kind < 0 || kind >= PCAS_K_COUNT || !launches || !total_ms)
        return fail(PCAS_ERR_INVALID_ARG, "bad profile query");
    std::lock_guard<std::mutex> lk(g_prof_mutex);
    *launches = g_launches[kind];
    double ms = 0.0;
    for (int i = 0; i < g_ev_used; i++) {
        if (g_ev_kind[i] != kind) continue;
        float t = 0.f;
        PCAS_CUDA(cudaEventSynchronize(g_ev[2 * i + 1]));
        PCAS_CUDA(cudaEventElapsedTime(&t, g_ev[2 * i], g_ev[2 * i + 1]));
        ms += t;
    }
    *total_ms = ms;
    return PCAS_OK;
}

const char* pcas_last_error(void) { return g_err; }

int pcas_version(void) { return PCAS_VERSION; }

size_t pcas_workspace_bytes(const pcas_vol* vol, const pcas_cb* cb, int K) {
    if (check_vol(vol) != PCAS_OK || !cb || cb->nu < 1 || cb->nv < 1 || K < 1 || K > PCAS_KMAX) return 0;
    return layout(vol, cb, K).total;
}

int pca_dvf(const float* mean, const float* U, int K, const double* w, const pcas_vol* vol,
            float* dvf, void* stream) {
    PCAS_TRY(check_vol(vol));
    PCAS_TRY(check_model(mean, U, K));
    PCAS_TRY(check_ptr(w, "w"));
    PCAS_TRY(check_ptr(dvf, "dvf"));
    PCAS_TRY(check_finite(w, K, "w"));
    float wf[PCAS_KMAX] = {0};
    for (int k = 0; k < K; k++) wf[k] = (float)w[k];
    cudaStream_t s = as_stream(stream);
    PCAS_LAUNCH(PCAS_K_PCA_DVF, s, launch_pca_dvf(mean, U, DT_F32, K, wf, make_grid(vol), dvf, s));
    return PCAS_OK;
}

int warp_volume(const float* f0, const float* dvf, const pcas_vol* vol, float* f, void* stream) {
    PCAS_TRY(check_vol(vol));
    PCAS_TRY(check_ptr(f0, "f0"));
    PCAS_TRY(check_ptr(dvf, "dvf"));
    PCAS_TRY(check_ptr(f, "f"));
    cudaStream_t s = as_stream(stream);
    PCAS_LAUNCH(PCAS_K_WARP_DVF, s, launch_warp_dvf(f0, DT_F32, dvf, make_grid(vol), f, s));
    return PCAS_OK;
}

int drr_forward(const float* f, const pcas_vol* vol, const pcas_cb* cb, double step_mm, float* p,
                void* stream) {
    PCAS_TRY(check_vol(vol));
    PCAS_TRY(check_ptr(f, "f"));
    PCAS_TRY(check_ptr(p, "p"));
    View V;
    PCAS_TRY(make_view(vol, cb, step_mm, &V));
    cudaStream_t s = as_stream(stream);
    PCAS_LAUNCH(PCAS_K_DRR, s, launch_drr_plain(f, make_grid(vol), V, p, s));
    return PCAS_OK;
}

int drr_siddon(const float* f, const pcas_vol* vol, const pcas_cb* cb, float* p, void* stream) {
    PCAS_TRY(check_vol(vol));
    PCAS_TRY(check_ptr(f, "f"));
    PCAS_TRY(check_ptr(p, "p"));
    View V;
    PCAS_TRY(make_view(vol, cb, 1.0, &V));        // geometry checks (volume ahead of the source)
    SidView D;
    const double sa = sin(cb->angle_rad), ca = cos(cb->angle_rad);
    const double S[3] = {cb->sad * sa, -cb->sad * ca, 0.0};
    const double ew[3] = {-sa, ca, 0.0}, eu[3] = {ca, sa, 0.0}, ev[3] = {0.0, 0.0, 1.0};
    for (int c = 0; c < 3; c++) { D.S[c] = S[c]; D.ew[c] = ew[c]; D.eu[c] = eu[c]; D.ev[c] = ev[c]; }
    D.sdd = cb->sdd;
    D.u0 = cb->off_u - 0.5 * (cb->nu - 1) * cb->du;
    D.v0 = cb->off_v - 0.5 * (cb->nv - 1) * cb->dv;
    D.du = cb->du;
    D.dv = cb->dv;
    D.o[0] = vol->ox; D.o[1] = vol->oy; D.o[2] = vol->oz;
    D.s[0] = vol->sx; D.s[1] = vol->sy; D.s[2] = vol->sz;
    D.n[0] = vol->nx; D.n[1] = vol->ny; D.n[2] = vol->nz;
    D.nu = cb->nu;
    D.nv = cb->nv;
    cudaStream_t s = as_stream(stream);
    PCAS_LAUNCH(PCAS_K_SIDDON, s, launch_drr_siddon(f, D, p, s));
    return PCAS_OK;
}

int drr_adjoint(const float* img, const pcas_vol* vol, const pcas_cb* cb, double step_mm, float* g,
                void* stream) {
    PCAS_TRY(check_vol(vol));
    PCAS_TRY(check_ptr(img, "img"));
    PCAS_TRY(check_ptr(g, "g"));
    View V;
    PCAS_TRY(make_view(vol, cb, step_mm, &V));
    cudaStream_t s = as_stream(stream);
    PCAS_LAUNCH(PCAS_K_ADJ, s, launch_adjoint_plain(img, make_grid(vol), V, g, s));
    return PCAS_OK;
}

int cost_grad_typed(const void* f0, const void* mean, const void* U, int dtype, int K, const double* w,
                    const float* y, const pcas_vol* vol, const pcas_cb* cb, double step_mm, double* J,
                    double* dJdw, double* ab, void* ws, size_t ws_bytes, void* stream) {
    PCAS_TRY(check_vol(vol));
    PCAS_TRY(check_model(mean, U, K));
    PCAS_TRY(check_dtype(dtype));
    PCAS_TRY(check_ptr(f0, "f0"));
    PCAS_TRY(check_ptr(y, "y"));
    PCAS_TRY(check_ptr(w, "w"));
    PCAS_TRY(check_ptr(J, "J"));
    PCAS_TRY(check_ptr(dJdw, "dJdw"));
    PCAS_TRY(check_ptr(ab, "ab"));
    PCAS_TRY(check_finite(w, K, "w"));
    View V;
    PCAS_TRY(make_view(vol, cb, step_mm, &V));
    const Tune T = tune_for(vol, cb, K, dtype);
    set_layouts(V, T, cb->angle_rad);
    Ws W;
    PCAS_TRY(bind_ws(ws, ws_bytes, vol, cb, K, &W));
    cudaStream_t s = as_stream(stream);
    Grid g = make_grid(vol);
    PCAS_CUDA(cudaMemsetAsync(W.fpad, 0, W.fpad_bytes, s));
    PCAS_TRY(launch_init(W.st, K, w, nullptr, s));
    PCAS_TRY(upload_view(W.view, V, s));
    PCAS_TRY(eval_gradient_pipeline(f0, mean, U, dtype, K, y, g, V, W, 0, T, s));
    SolveState h;
    PCAS_CUDA(cudaMemcpyAsync(&h, W.st, sizeof(h), cudaMemcpyDeviceToHost, s));
    PCAS_CUDA(cudaStreamSynchronize(s));
    if (h.phase == PH_SINGULAR) return fail(PCAS_ERR_SINGULAR, "Y^T Y is singular (constant image y)");
    *J = h.J;
    for (int k = 0; k < K; k++) dJdw[k] = h.G[k];
    ab[0] = h.a;
    ab[1] = h.b;
    return PCAS_OK;
}

int cost_grad(const float* f0, const float* mean, const float* U, int K, const double* w,
              const float* y, const pcas_vol* vol, const pcas_cb* cb, double step_mm, double* J,
              double* dJdw, double* ab, void* ws, size_t ws_bytes, void* stream) {
    return cost_grad_typed(f0, mean, U, PCAS_F32, K, w, y, vol, cb, step_mm, J, dJdw, ab, ws, ws_bytes, stream);
}

size_t pcas_workspace_bytes_f0(const pcas_vol* vol, const pcas_cb* cb, int K) {
    if (check_vol(vol) != PCAS_OK || !cb || cb->nu < 1 || cb->nv < 1 || K < 1 || K > PCAS_KMAX) return 0;
    const size_t N = (size_t)vol->nx * vol->ny * vol->nz;
    return layout(vol, cb, K).total + align256(N * sizeof(float)) + align256(N * 8) + 256;
}

int cost_grad_f0(const float* f0, const float* mean, const float* U, int K, const double* w,
                 const float* y, const pcas_vol* vol, const pcas_cb* cb, double step_mm, double* J,
                 double* dJdw, double* ab, float* dJdf0, void* ws, size_t ws_bytes, void* stream) {
    PCAS_TRY(check_vol(vol));
    PCAS_TRY(check_model(mean, U, K));
    PCAS_TRY(check_ptr(f0, "f0"));
    PCAS_TRY(check_ptr(y, "y"));
    PCAS_TRY(check_ptr(w, "w"));
    PCAS_TRY(check_ptr(J, "J"));
    PCAS_TRY(check_ptr(ab, "ab"));
    PCAS_TRY(check_finite(w, K, "w"));
    if (dJdf0 && !dJdw) return fail(PCAS_ERR_INVALID_ARG, "dJdf0 needs dJdw (the gradient passes run together)");
    View V;
    PCAS_TRY(make_view(vol, cb, step_mm, &V));
    const Tune T = tune_for(vol, cb, K, PCAS_F32);
    set_layouts(V, T, cb->angle_rad);
    if (!ws) return fail(PCAS_ERR_INVALID_ARG, "workspace is NULL");
    const size_t need = pcas_workspace_bytes_f0(vol, cb, K);
    if (ws_bytes < need) return fail(PCAS_ERR_INVALID_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, need);
    Ws W;
    const size_t base = layout(vol, cb, K).total;
    PCAS_TRY(bind_ws(ws, base, vol, cb, K, &W));
    const size_t N = (size_t)vol->nx * vol->ny * vol->nz;
    char* extra = static_cast<char*>(ws) + base;
    float* z = reinterpret_cast<float*>(extra);
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(extra + align256(N * sizeof(float)));
    unsigned int* zmax = reinterpret_cast<unsigned int*>(extra + align256(N * sizeof(float)) + align256(N * 8));
    cudaStream_t s = as_stream(stream);
    Grid g = make_grid(vol);
    PCAS_CUDA(cudaMemsetAsync(W.fpad, 0, W.fpad_bytes, s));
    PCAS_TRY(launch_init(W.st, K, w, nullptr, s));
    PCAS_TRY(upload_view(W.view, V, s));
    WSrc wsrc{};
    wsrc.dev = W.st->w;
    wsrc.phase = &W.st->phase;
    PCAS_TRY(stage_f0h(f0, DT_F32, g, W, T, s));
    if (dJdw)       // the gradient at w follows: its Jacobian pass comes with the warp
        PCAS_LAUNCH(PCAS_K_WARP_PCA, s, first_warp(W, T, g, mean, U, DT_F32, K, s));
    else
        PCAS_LAUNCH(PCAS_K_WARP_PCA, s, launch_warp_pca(W.f0h, mean, U, DT_F32, K, wsrc, g, W.view, W.fpad,
                                                        pair_of(W, T), W.st->box[0], occ_of(W, T), s));
    PCAS_LAUNCH(PCAS_K_DRR_SOLVER, s,
                launch_drr_solver(W.fpad, W.fpair, W.fpad4, g, V, W.view, y, W.pbuf, 0, W.st, W.part_drr, T, 0ull, 0,
                                  occ_of(W, T), s));
    PCAS_LAUNCH(PCAS_K_RESID, s, launch_resid(W.pbuf, y, V, W.view, 1, W.rayt, W.st, W.part_res, s));
    if (dJdw)
        PCAS_LAUNCH(PCAS_K_ADJ_GRAD, s,
                    launch_adjoint_grad(W.rayt, g, W.view, W.f0h, occ_of(W, T).f0m, mean, U, DT_F32, K, 0, W.st,
                                        W.part_adj, W.adj, T.vt, gather_blocks(T), 0ull, 0, nullptr, s));
    if (dJdf0)
        PCAS_LAUNCH(PCAS_K_GRAD_F0, s, launch_grad_f0(W.rayt, g, W.view, mean, U, K, W.st, z, zmax, acc, dJdf0, s));
    SolveState h;
    PCAS_CUDA(cudaMemcpyAsync(&h, W.st, sizeof(h), cudaMemcpyDeviceToHost, s));
    PCAS_CUDA(cudaStreamSynchronize(s));
    if (h.phase == PH_SINGULAR) return fail(PCAS_ERR_SINGULAR, "Y^T Y is singular (constant image y)");
    *J = h.J;
    if (dJdw)
        for (int k = 0; k < K; k++) dJdw[k] = h.G[k];
    ab[0] = h.a;
    ab[1] = h.b;
    return PCAS_OK;
}

int solve_projection_typed(const void* f0, const void* mean, const void* U, int dtype, int K,
                           const float* y, const pcas_vol* vol, const pcas_cb* cb, const double* w_init,
                           const pcas_params* prm, double* w_out, pcas_stats* stats, void* ws,
                           size_t ws_bytes, void* stream) {
    PCAS_TRY(check_vol(vol));
    PCAS_TRY(check_model(mean, U, K));
    PCAS_TRY(check_dtype(dtype));
    PCAS_TRY(check_ptr(f0, "f0"));
    PCAS_TRY(check_ptr(y, "y"));
    PCAS_TRY(check_ptr(w_init, "w_init"));
    PCAS_TRY(check_ptr(prm, "params"));
    PCAS_TRY(check_ptr(w_out, "w_out"));
    PCAS_TRY(check_finite(w_init, K, "w_init"));
    if (!(prm->mu0 > 0) || !(prm->alpha >= 0) || !(prm->beta > 0 && prm->beta < 1) ||
        !(prm->mu_min >= 0) || prm->max_iter < 0 || prm->max_trials < 0 || prm->max_trials > 1000)
        return fail(PCAS_ERR_INVALID_ARG, "solver parameters out of range");
    return solve_host(f0, mean, U, dtype, K, y, vol, cb, w_init, prm, tune_for(vol, cb, K, dtype), w_out, stats,
                      ws, ws_bytes, as_stream(stream));
}

int solve_projection(const float* f0, const float* mean, const float* U, int K, const float* y,
                     const pcas_vol* vol, const pcas_cb* cb, const double* w_init,
                     const pcas_params* prm, double* w_out, pcas_stats* stats, void* ws,
                     size_t ws_bytes, void* stream) {
    return solve_projection_typed(f0, mean, U, PCAS_F32, K, y, vol, cb, w_init, prm, w_out, stats, ws,
                                  ws_bytes, stream);
}

// ------------------------------------------------------------- autotuner
}  // extern "C"

namespace {

pcas_tuning to_public(const Tune& T) {
    pcas_tuning t;
    t.ray_lw1 = T.lw1; t.chunk1 = T.chunk1; t.voxel_tile = T.vt; t.gather_per_sm = T.adj_mult;
    t.skip_empty = T.skip;
    for (int b = 0; b < NBIN; b++) {
        t.ray_lw4[b] = T.lw4[b]; t.chunk[b] = T.chunk4[b]; t.swap[b] = T.swap[b];
    }
    return t;
}

int from_public(const pcas_tuning* t, Tune* T) {
    if (!t) return fail(PCAS_ERR_INVALID_ARG, "tuning is NULL");
    if (t->ray_lw1 < 2 || t->ray_lw1 > 4 || t->chunk1 < 0 || t->chunk1 > 128 || (t->chunk1 & 1) ||
        t->voxel_tile < 0 || t->voxel_tile >= NVOXTILE || t->gather_per_sm < 1 || t->gather_per_sm > 26 ||
        t->skip_empty < 0 || t->skip_empty > 1)
        return fail(PCAS_ERR_INVALID_ARG, "tuning field out of range");
    for (int b = 0; b < NBIN; b++)
        if (t->ray_lw4[b] < 2 || t->ray_lw4[b] > 4 || t->chunk[b] < 2 || t->chunk[b] > 64 || (t->chunk[b] & 1) ||
            t->swap[b] > 1)
            return fail(PCAS_ERR_INVALID_ARG, "tuning field of angle bin %d out of range", b);
    T->lw1 = t->ray_lw1; T->chunk1 = t->chunk1; T->vt = t->voxel_tile; T->adj_mult = t->gather_per_sm;
    T->skip = t->skip_empty;
    for (int b = 0; b < NBIN; b++) {
        T->lw4[b] = t->ray_lw4[b]; T->chunk4[b] = t->chunk[b]; T->swap[b] = t->swap[b];
    }
    return PCAS_OK;
}

// Runs one trial solve with shapes X at the centre angle of bin b and returns
// the mean event time per launch of each kernel class (0 where none ran).
struct Trial {
    const void *f0, *mean, *U;
    int dtype, K;
    const float* y;
    const pcas_vol* vol;
    const pcas_cb* cb;
    pcas_params prm;
    double w0[PCAS_KMAX];
    void* ws;
    size_t ws_bytes;
    cudaStream_t s;
    LocalTimer* timer;

    int run(const Tune& X, int b, double avg[PCAS_K_COUNT]) {
        for (int k = 0; k < PCAS_K_COUNT; k++) avg[k] = 0.0;
        pcas_cb c = *cb;
        c.angle_rad = b * (M_PI / NBIN);
        double w[PCAS_KMAX];
        pcas_stats st;
        timer->used = 0;
        t_local = timer;
        const int rc = solve_host(f0, mean, U, dtype, K, y, vol, &c, w0, &prm, X, w, &st, ws, ws_bytes, s);
        t_local = nullptr;
        if (rc != PCAS_OK) return rc;
        PCAS_CUDA(cudaStreamSynchronize(s));
        double tot[PCAS_K_COUNT] = {0};
        int n[PCAS_K_COUNT] = {0};
        for (int i = 0; i < timer->used; i++) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, timer->ev[2 * i], timer->ev[2 * i + 1]) != cudaSuccess) continue;
            tot[timer->kind[i]] += ms;
            n[timer->kind[i]]++;
        }
        for (int k = 0; k < PCAS_K_COUNT; k++) avg[k] = n[k] ? tot[k] / n[k] : 0.0;
        return PCAS_OK;
    }
};

}  // namespace

extern "C" {

int pcas_autotune(const void* f0, const void* mean, const void* U, int dtype, int K, const pcas_vol* vol,
                  const pcas_cb* cb, const pcas_params* params, const double* w_init, const float* y, void* ws,
                  size_t ws_bytes, pcas_tuning* out, void* stream) {
    PCAS_TRY(check_vol(vol));
    PCAS_TRY(check_model(mean, U, K));
    PCAS_TRY(check_dtype(dtype));
    PCAS_TRY(check_ptr(f0, "f0"));
    PCAS_TRY(check_ptr(y, "y"));
    PCAS_TRY(check_ptr(params, "params"));
    if (!cb) return fail(PCAS_ERR_INVALID_ARG, "cb is NULL");
    if (w_init) PCAS_TRY(check_finite(w_init, K, "w_init"));
    {
        View V;
        PCAS_TRY(make_view(vol, cb, params->step_mm, &V));
        Ws W;
        PCAS_TRY(bind_ws(ws, ws_bytes, vol, cb, K, &W));
    }
    Trial tr;
    tr.f0 = f0; tr.mean = mean; tr.U = U; tr.dtype = dtype; tr.K = K; tr.y = y; tr.vol = vol; tr.cb = cb;
    tr.prm = *params;
    if (tr.prm.max_iter > 3) tr.prm.max_iter = 3;
    for (int k = 0; k < PCAS_KMAX; k++) tr.w0[k] = (w_init && k < K) ? w_init[k] : 0.0;
    tr.ws = ws;
    tr.ws_bytes = ws_bytes;
    tr.s = as_stream(stream);
    LocalTimer* timer = new LocalTimer();
    tr.timer = timer;
    Tune best = tune_for(vol, cb, K, dtype);
    double a[PCAS_K_COUNT];
    int rc = PCAS_OK;
    bool ok_bin[NBIN];
    for (int b = 0; b < NBIN; b++) ok_bin[b] = true;
    const int probe[4] = {0, 2, 4, 6};
    // A shape replaces the one in place (the default, or the choice of an
    // earlier step) only when it is faster by more than this margin, and
    // among the shapes within the margin of the fastest the first in the
    // candidate list's order is taken: choices that timing noise would flip
    // from run to run -- and with them, through the order of the projectors'
    // and the gradient's sums, the rounding of the results -- stay put.
    const double keep = 0.985;
    auto sweep = [&](auto apply, const int* cands, int ncand, const int* kinds, int nkinds, const int* bins,
                     int nbins, int* choice) -> int {
        constexpr int kMaxCand = 8;
        if (ncand > kMaxCand) return fail(PCAS_ERR_INVALID_ARG, "autotune: too many candidates");
        double bestt = 0.0, inct = -1.0, tc[kMaxCand];
        bool any = false;
        const int inc = *choice;
        for (int c = 0; c < ncand; c++) {
            Tune X = best;
            apply(X, cands[c]);
            double t = 0.0;
            int used = 0;
            for (int q = 0; q < nbins; q++) {
                if (!ok_bin[bins[q]]) continue;
                const int r = tr.run(X, bins[q], a);
                if (r == PCAS_ERR_INVALID_ARG) { ok_bin[bins[q]] = false; continue; }   // view invalid here
                if (r != PCAS_OK) return r;
                for (int k = 0; k < nkinds; k++) t += a[kinds[k]];
                used++;
            }
            tc[c] = used ? t : -1.0;
            if (used && cands[c] == inc) inct = t;
            if (used && (!any || t < bestt)) bestt = t;
            any = any || used;
        }
        if (!any) return PCAS_OK;
        if (inct > 0.0 && bestt > keep * inct) return PCAS_OK;      // the incumbent stays
        for (int c = 0; c < ncand; c++)
            if (tc[c] > 0.0 && keep * tc[c] <= bestt) { *choice = cands[c]; break; }
        return PCAS_OK;
    };
    // 0. empty-space skipping, timed over the warps (which mark the bricks) and
    //    the projectors (which walk them)
    {
        const int onoff[2] = {1, 0};
        const int kw[4] = {PCAS_K_WARP_PCA, PCAS_K_DRR_SOLVER, PCAS_K_WARP_BATCH, PCAS_K_DRR_BATCH};
        int c = best.skip;
        rc = sweep([](Tune& X, int v) { X.skip = v; }, onoff, 2, kw, 4, probe, 4, &c);
        best.skip = c;
        for (int b = 0; b < NBIN; b++) ok_bin[b] = true;
    }
    // 1. per angle bin, the layout of the solver volumes, timed over every warp
    //    and projector kernel together (they write and read the same buffers)
    for (int b = 0; b < NBIN && rc == PCAS_OK; b++) {
        double tt[2] = {0, 0};
        for (int sw = 0; sw < 2 && ok_bin[b]; sw++) {
            Tune X = best;
            X.swap[b] = (unsigned char)sw;
            const int r = tr.run(X, b, a);
            if (r == PCAS_ERR_INVALID_ARG) { ok_bin[b] = false; break; }   // view invalid at this angle
            if (r != PCAS_OK) { rc = r; break; }
            tt[sw] = a[PCAS_K_WARP_PCA] + a[PCAS_K_DRR_SOLVER] + 2.0 * (a[PCAS_K_WARP_BATCH] + a[PCAS_K_DRR_BATCH]);
        }
        if (rc != PCAS_OK || !ok_bin[b]) continue;
        const int cur = best.swap[b] ? 1 : 0;
        if (tt[1 - cur] < keep * tt[cur]) best.swap[b] = (unsigned char)(1 - cur);
    }
    // 2. per angle bin, the patch width and chunk of the batch projector (the
    //    same rule: the incumbent, else the first within the margin)
    for (int b = 0; b < NBIN && rc == PCAS_OK; b++) {
        if (!ok_bin[b]) continue;
        const int chunks[3] = {12, 16, 24};
        double bestt = 0.0, inct = -1.0, tc[3][3];
        const int ilw = best.lw4[b], ich = best.chunk4[b];
        bool any = false;
        for (int lw = 2; lw <= 4 && rc == PCAS_OK; lw++) {
            for (int c = 0; c < 3 && rc == PCAS_OK; c++) {
                tc[lw - 2][c] = -1.0;
                Tune X = best;
                X.lw4[b] = (unsigned char)lw;
                X.chunk4[b] = (unsigned char)chunks[c];
                rc = tr.run(X, b, a);
                if (rc != PCAS_OK || a[PCAS_K_DRR_BATCH] <= 0.0) continue;
                const double t = a[PCAS_K_DRR_BATCH];
                tc[lw - 2][c] = t;
                if (lw == ilw && chunks[c] == ich) inct = t;
                if (!any || t < bestt) bestt = t;
                any = true;
            }
        }
        if (rc != PCAS_OK || !any || (inct > 0.0 && bestt > keep * inct)) continue;
        bool set = false;
        for (int lw = 2; lw <= 4 && !set; lw++)
            for (int c = 0; c < 3 && !set; c++)
                if (tc[lw - 2][c] > 0.0 && keep * tc[lw - 2][c] <= bestt) {
                    best.lw4[b] = (unsigned char)lw;
                    best.chunk4[b] = (unsigned char)chunks[c];
                    set = true;
                }
    }
    // 3. patch width and chunk of the one-volume projector (0: it reads through L1)
    if (rc == PCAS_OK) {
        const int lws[3] = {2, 3, 4};
        const int k1[1] = {PCAS_K_DRR_SOLVER};
        int c = best.lw1;
        rc = sweep([](Tune& X, int v) { X.lw1 = v; }, lws, 3, k1, 1, probe, 4, &c);
        best.lw1 = c;
    }
    if (rc == PCAS_OK) {
        const int ch1[3] = {0, 32, 64};
        const int k1[1] = {PCAS_K_DRR_SOLVER};
        int c = best.chunk1;
        rc = sweep([](Tune& X, int v) { X.chunk1 = v; }, ch1, 3, k1, 1, probe, 4, &c);
        best.chunk1 = c;
    }
    // 4. voxel tile and gather size of the gradient pass
    if (rc == PCAS_OK) {
        const int vts[NVOXTILE] = {0, 1, 2, 3, 4, 5}, gs[3] = {4, 8, 16};
        const int ka[1] = {PCAS_K_ADJ_GRAD};
        // the voxel tile also shapes the first evaluation's warp, which does
        // the first gradient's Jacobian pass
        const int kv[2] = {PCAS_K_WARP_PCA, PCAS_K_ADJ_GRAD};
        const int bins2[2] = {0, 4};
        int c = best.vt;
        rc = sweep([](Tune& X, int v) { X.vt = v; }, vts, NVOXTILE, kv, 2, probe, 4, &c);
        best.vt = c;
        int g = best.adj_mult;
        if (rc == PCAS_OK) rc = sweep([](Tune& X, int v) { X.adj_mult = v; }, gs, 3, ka, 1, bins2, 2, &g);
        best.adj_mult = g;
    }
    for (int i = 0; i < timer->created; i++) cudaEventDestroy(timer->ev[i]);
    delete timer;
    if (rc != PCAS_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tunes[bucket_of(vol, cb, K, dtype)] = best;
    }
    if (out) *out = to_public(best);
    return PCAS_OK;
}

int pcas_tuning_get(const pcas_vol* vol, const pcas_cb* cb, int K, int dtype, pcas_tuning* out) {
    PCAS_TRY(check_vol(vol));
    PCAS_TRY(check_ptr(out, "out"));
    if (!cb) return fail(PCAS_ERR_INVALID_ARG, "cb is NULL");
    *out = to_public(tune_for(vol, cb, K, dtype));
    return PCAS_OK;
}

int pcas_tuning_set(const pcas_vol* vol, const pcas_cb* cb, int K, int dtype, const pcas_tuning* t) {
    PCAS_TRY(check_vol(vol));
    if (!cb) return fail(PCAS_ERR_INVALID_ARG, "cb is NULL");
    Tune T;
    PCAS_TRY(from_public(t, &T));
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    g_tunes[bucket_of(vol, cb, K, dtype)] = T;
    return PCAS_OK;
}

int pcas_tuning_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    g_tunes.clear();
    return PCAS_OK;
}

// ---------------------------------------------------------------------------
// cost_grad_static: cost_grad for callers that cannot allocate device memory
// (real-time loops where an allocation could stall, or host programs whose own
// allocator owns all device memory).  Its scratch is the file-scope array
// below instead of a caller workspace.
}  // extern "C"

namespace {

__device__ __align__(256) unsigned char g_static_scratch[PCAS_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 256;
std::mutex g_static_mutex;
void* g_static_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device, looked up once
// per device.  In host code the symbol itself is only a host-side stand-in.
int static_scratch(void** out) {
    int dev = 0;
    PCAS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(PCAS_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_static_mutex);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        PCAS_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return PCAS_OK;
}

}  // namespace

extern "C" {

int cost_grad_static(const float* f0, const float* mean, const float* U, int K, const double* w,
                     const float* y, const pcas_vol* vol, const pcas_cb* cb, double step_mm,
                     double* J, double* dJdw, double* ab, void* stream) {
    PCAS_TRY(check_vol(vol));
    if (!cb || cb->nu < 1 || cb->nv < 1) return fail(PCAS_ERR_INVALID_ARG, "detector size invalid");
    const size_t need = layout(vol, cb, K < 1 ? 1 : K > PCAS_KMAX ? PCAS_KMAX : K).total;
    if (need > (size_t)PCAS_STATIC_SCRATCH_BYTES)
        return fail(PCAS_ERR_INVALID_ARG,
                    "cost_grad_static: this volume and detector need %zu bytes of scratch, more than the "
                    "%d-byte static scratch; use cost_grad with a caller workspace",
                    need, PCAS_STATIC_SCRATCH_BYTES);
    void* scratch = nullptr;
    PCAS_TRY(static_scratch(&scratch));
    return cost_grad(f0, mean, U, K, w, y, vol, cb, step_mm, J, dJdw, ab, scratch,
                     (size_t)PCAS_STATIC_SCRATCH_BYTES, stream);
}

int localize_tumor_typed(const void* mean, const void* U, int dtype, int K, const double* w,
                         const pcas_vol* vol, const double c_ref[3], int max_iter, double tol_mm,
                         double c_out[3], void* stream) {
    PCAS_TRY(check_vol(vol));
    PCAS_TRY(check_model(mean, U, K));
    PCAS_TRY(check_dtype(dtype));
    PCAS_TRY(check_ptr(w, "w"));
    PCAS_TRY(check_ptr(c_ref, "c_ref"));
    PCAS_TRY(check_ptr(c_out, "c_out"));
    PCAS_TRY(check_finite(w, K, "w"));
    PCAS_TRY(check_finite(c_ref, 3, "c_ref"));
    if (max_iter < 1 || max_iter > 100000 || !(tol_mm > 0))
        return fail(PCAS_ERR_INVALID_ARG, "max_iter must be in [1, 1e5] and tol_mm > 0");
    double wv[PCAS_KMAX] = {0};
    for (int k = 0; k < K; k++) wv[k] = w[k];
    cudaStream_t s = as_stream(stream);
    // The 32-byte result lands in a file-scope device slot and is copied out
    // before the call returns; a host mutex keeps concurrent callers apart.
    std::lock_guard<std::mutex> lock(g_localize_mutex);
    double* out = nullptr;
    PCAS_CUDA(cudaGetSymbolAddress((void**)&out, d_localize_out));
#define PCAS_LOC(T)                                                                                  \
    PCAS_LAUNCH(PCAS_K_LOCALIZE, s,                                                                  \
                (k_localize<T><<<1, 32, 0, s>>>(static_cast<const T*>(mean), static_cast<const T*>(U), \
                                                K, make_grid(vol), wv[0], wv[1], wv[2], wv[3], wv[4],  \
                                                wv[5], wv[6], wv[7], vol->ox, vol->oy, vol->oz,        \
                                                1.0 / vol->sx, 1.0 / vol->sy, 1.0 / vol->sz, c_ref[0], \
                                                c_ref[1], c_ref[2], max_iter, tol_mm, out),            \
                 cudaGetLastError()))
    if (dtype == PCAS_F32) PCAS_LOC(float);
    else if (dtype == PCAS_BF16) PCAS_LOC(__nv_bfloat16);
    else PCAS_LOC(__half);
#undef PCAS_LOC
    double h[4];
    PCAS_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
    PCAS_CUDA(cudaStreamSynchronize(s));
    c_out[0] = h[0]; c_out[1] = h[1]; c_out[2] = h[2];
    return h[3] != 0.0 ? PCAS_OK : PCAS_NOT_CONVERGED;
}

int localize_tumor(const float* mean, const float* U, int K, const double* w, const pcas_vol* vol,
                   const double c_ref[3], int max_iter, double tol_mm, double c_out[3],
                   void* stream) {
    return localize_tumor_typed(mean, U, PCAS_F32, K, w, vol, c_ref, max_iter, tol_mm, c_out, stream);
}

// Eq. (3) fit, host: per coefficient, normal equations of the order-L
// least-squares predictor, Cholesky-free Gaussian elimination with pivoting.
int lp_fit(const double* trace, int T, int K, int L, double* c) {
    if (!trace || !c) return fail(PCAS_ERR_INVALID_ARG, "trace and c must be non-NULL");
    if (K < 1 || L < 1 || L > 16 || T <= 2 * L)
        return fail(PCAS_ERR_INVALID_ARG, "need K >= 1, 1 <= L <= 16 and T > 2L");
    for (int k = 0; k < K; k++) {
        double A[16][17];
        memset(A, 0, sizeof(A));
        for (int t = L; t < T; t++) {
            double xt = trace[(long)t * K + k];
            for (int a = 0; a < L; a++) {
                double xa = trace[(long)(t - 1 - a) * K + k];
                A[a][L] += xa * xt;
                for (int b = 0; b < L; b++) A[a][b] += xa * trace[(long)(t - 1 - b) * K + k];
            }
        }
        for (int col = 0; col < L; col++) {
            int piv = col;
            for (int r = col + 1; r < L; r++)
                if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
            if (A[piv][col] == 0.0) return fail(PCAS_ERR_SINGULAR, "prediction normal equations singular");
            if (piv != col)
                for (int j = 0; j <= L; j++) {
                    double t = A[col][j];
                    A[col][j] = A[piv][j];
                    A[piv][j] = t;
                }
            for (int r = col + 1; r < L; r++) {
                double f = A[r][col] / A[col][col];
                for (int j = col; j <= L; j++) A[r][j] -= f * A[col][j];
            }
        }
        for (int r = L - 1; r >= 0; r--) {
            double acc = A[r][L];
            for (int j = r + 1; j < L; j++) acc -= A[r][j] * c[k * L + j];
            c[k * L + r] = acc / A[r][r];
        }
    }
    return PCAS_OK;
}

int lp_predict(const double* hist, const double* c, int K, int L, double* w0) {
    if (!hist || !c || !w0) return fail(PCAS_ERR_INVALID_ARG, "hist, c and w0 must be non-NULL");
    if (K < 1 || L < 1) return fail(PCAS_ERR_INVALID_ARG, "need K >= 1 and L >= 1");
    for (int k = 0; k < K; k++) {          // fused multiply-adds in l order (as the device warm start)
        double acc = 0.0;
        for (int l = 0; l < L; l++) acc = fma(c[k * L + l], hist[(long)l * K + k], acc);
        w0[k] = acc;
    }
    return PCAS_OK;
}

}  // extern "C"

// ===========================================================================
// Device-driven solve: the loop of the Appendix as one CUDA graph.  Two nested
// conditional WHILE nodes replace the host loop -- iterations, and candidate
// batches inside an iteration.  The gradient's last block opens the batch
// loop, the batch projector's last block decides each batch and whether
// another follows, and a one-thread controller ends each iteration; every one
// of these sets its condition on every path out.  Both loops are bounded by construction:
// an iteration either accepts a step (at most max_iter of them) or ends the
// solve, and every batch tries at least one step size of the iteration's
// schedule (at most max_trials).  The view and the initial coefficients are
// copied in before each launch from a ring of pinned host slots, so one
// instantiated graph serves every gantry angle, and launches can be queued
// ahead.  In a run of consecutive projections (pcas_solver_seq_*) the warm
// start of Eq. (3) is taken on the device from the solutions kept there, and
// the tumour localisation of Sec. II.A follows each solve on a stream of its
// own (it overlaps the next projection's solve, which does not need it):
// projection after projection goes by without a host round trip.
// ===========================================================================
namespace {

struct InitBlock {
    double w[PCAS_KMAX];
    double mu0, alpha, beta, mu_min;
    int K, max_trials, max_iter;
    int seq;                  // 1: start from the run's history (Eq. 3), localise at the end
    int slot;                 // ring slot of this launch (a run's result record)
};

// Per-launch staging (view + start), one device copy and SEQ_RING host slots.
struct Stage {
    View v;
    InitBlock ib;
};

enum { LP_MAX = 8, SEQ_RING = 64 };

// A run of consecutive projections: the Eq. (3) predictor, the localisation
// parameters, and the solutions so far (hist[0] the latest).
struct SeqBlock {
    double lp[PCAS_KMAX * LP_MAX];    // c[k * L + l] as lp_fit
    double c_ref[3], loc_tol;
    double o[3], is[3];               // volume origin and reciprocal spacing
    int L, loc_max_iter;
    int n;                            // solutions in the history (n >= L: full predictor)
    int f0_ready;                     // the run's first projection has copied the reference CT
    double hist[LP_MAX][PCAS_KMAX];
};

// Result of one projection of a run (a ring of SEQ_RING on the device, one per
// slot), copied to the host slot after the localisation.
struct SeqOut {
    double w[PCAS_KMAX];
    double c[4];                      // centroid (mm) and 1 if the fixed point converged
    double J0, J, a, b, mu;
    int iters, evals, phase, launches;
};

// Eq. (3) on the device: w0 = sum_l c[k][l] w*(t-1-l) with fused
// multiply-adds in l order, exactly as the host lp_predict.  Before L
// solutions exist the run starts from the latest one (or from ib->w first).
__device__ double seq_start(const SeqBlock* sq, const InitBlock* ib, int k) {
    const int n = sq->n, L = sq->L;
    if (n == 0) return ib->w[k];
    if (n < L) return sq->hist[0][k];
    double acc = 0.0;
    for (int l = 0; l < L; l++) acc = fma(sq->lp[k * L + l], sq->hist[l][k], acc);
    return acc;
}

__global__ void k_init_dev(SolveState* st, const InitBlock* __restrict__ ib, const SeqBlock* __restrict__ sq) {
    if (threadIdx.x != 0) return;
    st->keep_f0h = ib->seq && sq->f0_ready;   // a run reads the reference CT once
    for (int k = 0; k < PCAS_KMAX; k++) {
        st->w[k] = k < ib->K ? (ib->seq ? seq_start(sq, ib, k) : ib->w[k]) : 0.0;
        st->d[k] = 0.0;
        st->G[k] = 0.0;
        for (int j = 0; j < TRIAL_BATCH; j++) st->wt[j][k] = st->w[k];
    }
    for (int j = 0; j < TRIAL_BATCH; j++) st->mu_batch[j] = 0.0;
    st->gnorm = st->a = st->b = st->J = st->J0 = st->Jt = 0.0;
    st->mu = ib->mu0;
    for (int i = 0; i < NBUF; i++)
        for (int j = 0; j < NMOM; j++) st->mom[i][j] = 0.0;
    st->mu0 = ib->mu0; st->alpha = ib->alpha; st->beta = ib->beta; st->mu_min = ib->mu_min;
    st->K = ib->K; st->max_trials = ib->max_trials; st->max_iter = ib->max_iter;
    st->cur = 0; st->phase = PH_RUNNING; st->evals = 0; st->trials = 0;
    st->nvalid = 0; st->iters = 0; st->batches = 0; st->launches = 1;
    st->wide = 1;
    st->jac_ready = 0;
    for (int i = 0; i < 4; i++) st->counter[i] = 0u;
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 6; j++) st->box[i][j] = BOX_EMPTY;
}

// After the first evaluation (init, copy of f0, warp, projection, this kernel).
__global__ void k_ctrl_start(SolveState* st, cudaGraphConditionalHandle h_outer) {
    st->launches += 5;
    cudaGraphSetConditional(h_outer, (st->max_iter > 0 && st->phase < PH_STOP) ? 1u : 0u);
}

// End of an iteration (residual, three gradient kernels -- the last of which
// opened the batch loop -- the batches, and this kernel).
__global__ void k_ctrl_iter_end(SolveState* st, cudaGraphConditionalHandle h_outer) {
    st->launches += 5;
    int ph = st->phase;
    if (ph == PH_RUNNING) {          // batch cap reached without a decision: end the solve
        ph = PH_STOP;
        st->phase = ph;
    }
    if (ph == PH_ACCEPT || ph == PH_STOP) st->iters += 1;
    const bool more = ph == PH_ACCEPT && st->iters < st->max_iter;
    cudaGraphSetConditional(h_outer, more ? 1u : 0u);
}

// End of a device-driven solve (one warp).  In a run: the tumour centroid at
// the solution (Sec. II.A, the same fixed point as localize_tumor), the
// solution pushed onto the history, and the result record.
__global__ void k_seq_end(SolveState* st, const InitBlock* __restrict__ ib, SeqBlock* sq, SeqOut* out_ring) {
    if (threadIdx.x != 0) return;
    if (!ib->seq) {
        st->launches += 1;
        return;
    }
    double w[PCAS_KMAX];
    for (int k = 0; k < PCAS_KMAX; k++) w[k] = st->w[k];
    for (int l = LP_MAX - 1; l > 0; l--)
        for (int k = 0; k < PCAS_KMAX; k++) sq->hist[l][k] = sq->hist[l - 1][k];
    for (int k = 0; k < PCAS_KMAX; k++) sq->hist[0][k] = w[k];
    if (sq->n < LP_MAX) sq->n += 1;
    sq->f0_ready = 1;
    st->launches += 1;
    SeqOut* out = out_ring + ib->slot;
    for (int k = 0; k < PCAS_KMAX; k++) out->w[k] = w[k];
    out->J0 = st->J0; out->J = st->J; out->a = st->a; out->b = st->b; out->mu = st->mu;
    out->iters = st->iters; out->evals = st->evals; out->phase = st->phase; out->launches = st->launches;
}

// The tumour centroid at a run's solution (Sec. II.A, the same fixed point as
// localize_tumor), into the projection's result record.  Launched after the
// solve on the solver's localisation stream; reads only the run's constant
// parameters and the record's own coefficients.
template <typename T>
__global__ void k_seq_loc(const SeqBlock* __restrict__ sq, SeqOut* out, const T* __restrict__ mean,
                          const T* __restrict__ U, int K, Grid g) {
    double w[PCAS_KMAX];
    for (int k = 0; k < PCAS_KMAX; k++) w[k] = out->w[k];
    localize_warp(mean, U, K, g, w, sq->o[0], sq->o[1], sq->o[2], sq->is[0], sq->is[1], sq->is[2],
                  sq->c_ref[0], sq->c_ref[1], sq->c_ref[2], sq->loc_max_iter, sq->loc_tol, out->c);
    if (threadIdx.x == 0) out->launches += 1;
}

#define PCAS_G(call)                                                                              \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            cudaGraph_t g_junk;                                                                   \
            cudaStreamEndCapture(cs, &g_junk);                                                    \
            return fail(PCAS_ERR_CUDA, "graph build: %s failed: %s", #call, cudaGetErrorString(e_)); \
        }                                                                                         \
    } while (0)

// Adds a WHILE node after the current capture position and moves the capture past it.
int add_while(cudaStream_t cs, cudaGraphConditionalHandle h, cudaGraph_t* body) {
    cudaStreamCaptureStatus status;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    PCAS_G(cudaStreamGetCaptureInfo(cs, &status, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    PCAS_G(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp));
    *body = cp.conditional.phGraph_out[0];
    PCAS_G(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return PCAS_OK;
}

}  // namespace

struct pcas_solver_s {
    int device;
    pcas_vol vol;
    pcas_cb cb;
    pcas_params prm;
    int K, dtype;
    const void *f0, *mean, *U;
    Ws W;
    float* y;             // device, M floats (in the workspace)
    Stage* d_stage;       // device (in the workspace): view + start of the next launch
    SeqBlock* d_seq;      // device: the run of consecutive projections
    SeqOut* d_out;        // device [SEQ_RING]: results of a run, by slot
    Stage* h_ring;        // pinned host [SEQ_RING]: staging per launch
    SeqOut* h_out;        // pinned host [SEQ_RING]: results of a run
    SeqBlock* h_seq;      // pinned host: run parameters on their way to the device
    cudaEvent_t ev[SEQ_RING];   // a slot is free again once its launch passed this
    cudaEvent_t ev_solved[SEQ_RING];  // a run's solve of the slot is done (localisation may start)
    cudaStream_t loc_stream;          // localisations of a run's projections
    // host images of a run: uploaded on the copy stream into one of two
    // staging buffers (device, in the workspace) while earlier projections
    // solve, then copied device to device into y ahead of their own solve
    float* ystage[2];
    cudaStream_t cp_stream;
    cudaEvent_t ev_cp[2];             // the upload into ystage[b] is done
    cudaEvent_t ev_used[2];           // the solve stream has copied ystage[b] out
    int ynext;
    long long next;       // tickets handed out (slot = ticket % SEQ_RING)
    long long seq_first;  // first ticket of the current run (-1: no run)
    long long slot_ticket[SEQ_RING];  // ticket of a run's projection in each slot (-1: none)
    bool slot_counted[SEQ_RING];      // its launches already added to the profile
    SolveState* h_state;
    cudaGraphConditionalHandle h_outer, h_inner;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    View view0;           // geometry at creation (grid sizes)
    Tune tune;            // launch shapes of the size bucket at creation (captured)
    int layout;           // swap of the last staged view; -1: buffers all zero
    // fixed-view cache of P^T (caller memory; pcas_solver_fix_view): used by
    // the solves staged at exactly this angle and the creation offsets
    int pt_on;
    double pt_angle;
    const short4* pt_rect;
    const unsigned long long* pt_off;
    const float* pt_w;
};

struct pcas_batch_s {
    std::vector<pcas_solver> solvers;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace {

size_t solver_extra(const pcas_cb* cb) {
    const size_t img = align256((size_t)cb->nu * cb->nv * sizeof(float));
    return img + align256(sizeof(Stage)) + align256(sizeof(SeqBlock)) + align256(SEQ_RING * sizeof(SeqOut)) +
           2 * img;                       // the image, ..., and two staging images of a run
}

// Captures one device-driven solve into `graph` as an independent branch
// (optionally preceded by a copy of the measured image from y_src).
// A second capture stream and the two events of the residual branch (freed on
// every path out of capture_solve).
struct SideBranch {
    cudaStream_t cs2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaError_t init() {
        cudaError_t e = cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
        return e;
    }
    ~SideBranch() {
        if (join) cudaEventDestroy(join);
        if (fork) cudaEventDestroy(fork);
        if (cs2) cudaStreamDestroy(cs2);
    }
};

int capture_solve(pcas_solver s, cudaGraph_t graph, cudaStream_t cs, const float* y_src) {
    SideBranch side;
    if (side.init() != cudaSuccess) return fail(PCAS_ERR_CUDA, "graph build: stream/event creation failed");
    cudaStream_t cs2 = side.cs2;
    cudaEvent_t ev_fork = side.fork, ev_join = side.join;
    const Grid g = make_grid(&s->vol);
    const Ws& W = s->W;
    const View& V = s->view0;
    const size_t M = (size_t)s->cb.nu * s->cb.nv;
    PCAS_G(cudaGraphConditionalHandleCreate(&s->h_outer, graph, 0, cudaGraphCondAssignDefault));
    // prologue
    PCAS_G(cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    if (y_src) PCAS_G(cudaMemcpyAsync(s->y, y_src, M * sizeof(float), cudaMemcpyDeviceToDevice, cs));
    k_init_dev<<<1, 32, 0, cs>>>(W.st, &s->d_stage->ib, s->d_seq);
    PCAS_G(cudaGetLastError());
    const Occ oc = occ_of(W, s->tune);
    // the reference CT is copied for every solve, except after the first
    // projection of a run (k_init_dev sets keep_f0h then)
    PCAS_G(launch_fill_f0h(s->f0, s->dtype, g, W.f0h, s->tune.skip ? W.f0m : nullptr, &W.st->keep_f0h, cs));
    PCAS_G(first_warp(W, s->tune, g, s->mean, s->U, s->dtype, s->K, cs));
    PCAS_G(launch_drr_solver(W.fpad, W.fpair, W.fpad4, g, V, W.view, s->y, W.pbuf, 0, W.st, W.part_drr, s->tune, 0ull, 0,
                             oc, cs));
    k_ctrl_start<<<1, 1, 0, cs>>>(W.st, s->h_outer);
    PCAS_G(cudaGetLastError());
    cudaGraph_t outer_body;
    PCAS_TRY(add_while(cs, s->h_outer, &outer_body));
    k_seq_end<<<1, 32, 0, cs>>>(W.st, &s->d_stage->ib, s->d_seq, s->d_out);
    PCAS_G(cudaGetLastError());
    cudaGraph_t done;
    PCAS_G(cudaStreamEndCapture(cs, &done));
    // one iteration: residual + gradient, then the candidate batches
    PCAS_G(cudaGraphConditionalHandleCreate(&s->h_inner, outer_body, 0, cudaGraphCondAssignDefault));
    PCAS_G(cudaStreamBeginCaptureToGraph(cs, outer_body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    // residual (ray table) on a side branch beside the Jacobian pass; the gather joins both
    PCAS_G(cudaEventRecord(ev_fork, cs));
    PCAS_G(cudaStreamWaitEvent(cs2, ev_fork, 0));
    PCAS_G(launch_resid(W.pbuf, s->y, V, W.view, -1, W.rayt, W.st, W.part_res, cs2));
    PCAS_G(cudaEventRecord(ev_join, cs2));
    PCAS_G(launch_adjoint_grad(W.rayt, g, W.view, W.f0h, oc.f0m, s->mean, s->U, s->dtype, s->K, 1, W.st, W.part_adj,
                               W.adj, s->tune.vt, gather_blocks(s->tune), s->h_inner, 1, ev_join, cs));
    cudaGraph_t inner_body;
    PCAS_TRY(add_while(cs, s->h_inner, &inner_body));
    k_ctrl_iter_end<<<1, 1, 0, cs>>>(W.st, s->h_outer);
    PCAS_G(cudaGetLastError());
    PCAS_G(cudaStreamEndCapture(cs, &done));
    // one candidate batch: warp and projection; the projection's last block
    // decides the batch and whether another follows
    PCAS_G(cudaStreamBeginCaptureToGraph(cs, inner_body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    PCAS_G(launch_warp_batch(W.f0h, s->mean, s->U, s->dtype, s->K, W.st, g, W.view, W.fpad4, W.fpad, oc, cs));
    PCAS_G(launch_drr_solver(W.fpad, W.fpair, W.fpad4, g, V, W.view, s->y, W.pbuf, TRIAL_BATCH, W.st, W.part_drr,
                             s->tune, s->h_inner, 1, oc, cs));
    PCAS_G(cudaStreamEndCapture(cs, &done));
    return PCAS_OK;
}

#undef PCAS_G

// Takes the next staging slot (waiting until the launch that last used it
// has passed it) and returns its index; the ticket is s->next - 1.
int solver_slot(pcas_solver s, int* slot) {
    const int i = (int)(s->next % SEQ_RING);
    if (s->next >= SEQ_RING) PCAS_CUDA(cudaEventSynchronize(s->ev[i]));
    s->slot_ticket[i] = -1;               // its previous result, if any, is gone
    s->next += 1;
    *slot = i;
    return PCAS_OK;
}

// Stages the view of this angle and the start of a solve in a ring slot and
// enqueues its copy to the device (plus the zeroing of the solver volumes
// when the layout changes).  seq: start from the run's history instead of
// w_init (which is then only used for the run's first projection, may be NULL).
int solver_stage(pcas_solver s, double angle_rad, double off_u, double off_v, const double* w_init, int seq,
                 int* slot_out, cudaStream_t st) {
    pcas_cb cb = s->cb;
    cb.angle_rad = angle_rad;
    cb.off_u = off_u;
    cb.off_v = off_v;
    View V;
    PCAS_TRY(make_view(&s->vol, &cb, s->prm.step_mm, &V));
    if (w_init) PCAS_TRY(check_finite(w_init, s->K, "w_init"));
    else if (!seq) return fail(PCAS_ERR_INVALID_ARG, "w_init is NULL");
    set_layouts(V, s->tune, angle_rad);
    if (s->pt_on && angle_rad == s->pt_angle && off_u == s->cb.off_u && off_v == s->cb.off_v) {
        V.pt_rect = s->pt_rect;           // the fixed view: the gather reads the cached P^T
        V.pt_off = s->pt_off;
        V.pt_w = s->pt_w;
    }
    int slot;
    PCAS_TRY(solver_slot(s, &slot));
    const int lay = V.swap;
    if (s->layout >= 0 && s->layout != lay)   // the other layout's voxels lie on this one's halo
        PCAS_CUDA(cudaMemsetAsync(s->W.fpad, 0, s->W.fpad_bytes + s->W.fpad4_bytes, st));
    s->layout = lay;
    Stage& h = s->h_ring[slot];
    h.v = V;
    InitBlock ib = {};
    for (int k = 0; k < s->K; k++) ib.w[k] = w_init ? w_init[k] : 0.0;
    ib.mu0 = s->prm.mu0; ib.alpha = s->prm.alpha; ib.beta = s->prm.beta; ib.mu_min = s->prm.mu_min;
    ib.K = s->K; ib.max_trials = s->prm.max_trials; ib.max_iter = s->prm.max_iter;
    ib.seq = seq;
    ib.slot = slot;
    h.ib = ib;
    PCAS_CUDA(cudaMemcpyAsync(s->d_stage, &h, sizeof(Stage), cudaMemcpyHostToDevice, st));
    if (slot_out) *slot_out = slot;
    return PCAS_OK;
}

int solver_collect(pcas_solver s, double* w_out, pcas_stats* stats) {
    const SolveState& h = *s->h_state;
    if (h.phase == PH_SINGULAR) return fail(PCAS_ERR_SINGULAR, "Y^T Y is singular (constant image y)");
    if (w_out)
        for (int k = 0; k < s->K; k++) w_out[k] = h.w[k];
    if (stats) {
        stats->iters = h.iters;
        stats->evals = h.evals;
        stats->status = PCAS_OK;
        stats->J0 = h.J0;
        stats->J = h.J;
        stats->a = h.a;
        stats->b = h.b;
        stats->mu_last = h.mu;
    }
    return PCAS_OK;
}

void solver_free(pcas_solver s) {
    if (!s) return;
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    if (s->loc_stream) {
        cudaStreamSynchronize(s->loc_stream);
        cudaStreamDestroy(s->loc_stream);
    }
    if (s->cp_stream) {
        cudaStreamSynchronize(s->cp_stream);
        cudaStreamDestroy(s->cp_stream);
    }
    for (int i = 0; i < SEQ_RING; i++) {
        if (s->ev[i]) cudaEventDestroy(s->ev[i]);
        if (s->ev_solved[i]) cudaEventDestroy(s->ev_solved[i]);
    }
    for (int b = 0; b < 2; b++) {
        if (s->ev_cp[b]) cudaEventDestroy(s->ev_cp[b]);
        if (s->ev_used[b]) cudaEventDestroy(s->ev_used[b]);
    }
    if (s->h_ring) cudaFreeHost(s->h_ring);
    if (s->h_out) cudaFreeHost(s->h_out);
    if (s->h_seq) cudaFreeHost(s->h_seq);
    if (s->h_state) cudaFreeHost(s->h_state);
    delete s;
}

}  // namespace

extern "C" {

size_t pcas_solver_workspace_bytes(const pcas_vol* vol, const pcas_cb* cb, int K) {
    if (check_vol(vol) != PCAS_OK || !cb || cb->nu < 1 || cb->nv < 1 || K < 1 || K > PCAS_KMAX) return 0;
    return layout(vol, cb, K).total + solver_extra(cb);
}

int pcas_solver_create(pcas_solver* out, const void* f0, const void* mean, const void* U, int dtype, int K,
                       const pcas_vol* vol, const pcas_cb* cb, const pcas_params* prm, void* ws,
                       size_t ws_bytes, void* stream) {
    PCAS_TRY(check_ptr(out, "out"));
    *out = nullptr;
    PCAS_TRY(check_vol(vol));
    PCAS_TRY(check_model(mean, U, K));
    PCAS_TRY(check_dtype(dtype));
    PCAS_TRY(check_ptr(f0, "f0"));
    PCAS_TRY(check_ptr(prm, "params"));
    if (!(prm->mu0 > 0) || !(prm->alpha >= 0) || !(prm->beta > 0 && prm->beta < 1) || !(prm->mu_min >= 0) ||
        prm->max_iter < 0 || prm->max_iter > 100000 || prm->max_trials < 0 || prm->max_trials > 1000)
        return fail(PCAS_ERR_INVALID_ARG, "solver parameters out of range");
    View V;
    PCAS_TRY(make_view(vol, cb, prm->step_mm, &V));
    const size_t need = pcas_solver_workspace_bytes(vol, cb, K);
    if (!ws) return fail(PCAS_ERR_INVALID_ARG, "workspace is NULL");
    if (ws_bytes < need) return fail(PCAS_ERR_INVALID_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, need);
    const size_t base = layout(vol, cb, K).total;
    pcas_solver s = new pcas_solver_s();
    s->vol = *vol; s->cb = *cb; s->prm = *prm; s->K = K; s->dtype = dtype;
    s->f0 = f0; s->mean = mean; s->U = U; s->view0 = V; s->layout = -1;
    s->tune = tune_for(vol, cb, K, dtype);
    set_layouts(s->view0, s->tune, cb->angle_rad);
    int rc = bind_ws(ws, base, vol, cb, K, &s->W);
    if (rc != PCAS_OK) { solver_free(s); return rc; }
    char* extra = static_cast<char*>(ws) + base;
    size_t off = align256((size_t)cb->nu * cb->nv * sizeof(float));
    s->y = reinterpret_cast<float*>(extra);
    s->d_stage = reinterpret_cast<Stage*>(extra + off);
    off += align256(sizeof(Stage));
    s->d_seq = reinterpret_cast<SeqBlock*>(extra + off);
    off += align256(sizeof(SeqBlock));
    s->d_out = reinterpret_cast<SeqOut*>(extra + off);
    off += align256(SEQ_RING * sizeof(SeqOut));
    for (int b = 0; b < 2; b++) {
        s->ystage[b] = reinterpret_cast<float*>(extra + off);
        off += align256((size_t)cb->nu * cb->nv * sizeof(float));
    }
    s->W.view = &s->d_stage->v;           // the kernels read the staged view
    s->seq_first = -1;
    for (int i = 0; i < SEQ_RING; i++) s->slot_ticket[i] = -1;
    cudaStream_t st = as_stream(stream);
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->h_ring, SEQ_RING * sizeof(Stage), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->h_out, SEQ_RING * sizeof(SeqOut), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->h_seq, sizeof(SeqBlock), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->h_state, sizeof(SolveState), cudaHostAllocDefault);
    for (int i = 0; i < SEQ_RING && e == cudaSuccess; i++) {
        e = cudaEventCreateWithFlags(&s->ev[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_solved[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->loc_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cp_stream, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; b++) {
        e = cudaEventCreateWithFlags(&s->ev_cp[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_used[b], cudaEventDisableTiming);
    }
    // zero the halos once: the warp kernels never write them
    if (e == cudaSuccess) e = cudaMemsetAsync(s->W.fpad, 0, s->W.fpad_bytes + s->W.fpad4_bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->W.f0h, 0, s->W.f0h_bytes, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaGraphCreate(&s->graph, 0);
    if (e != cudaSuccess) {
        if (cs) cudaStreamDestroy(cs);
        solver_free(s);
        return fail(PCAS_ERR_CUDA, "solver set-up failed: %s", cudaGetErrorString(e));
    }
    rc = capture_solve(s, s->graph, cs, nullptr);
    cudaStreamDestroy(cs);
    if (rc != PCAS_OK) { solver_free(s); return rc; }
    e = cudaGraphInstantiate(&s->exec, s->graph, 0);
    if (e != cudaSuccess) {
        solver_free(s);
        return fail(PCAS_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    *out = s;
    return PCAS_OK;
}

float* pcas_solver_y_buffer(pcas_solver s) { return s ? s->y : nullptr; }

}  // extern "C"

namespace {

// Layout of a fixed-view cache of total footprint entries `total` for N voxels.
struct PtLayout {
    size_t off, rect, w, err, bytes;
};
PtLayout pt_layout(long N, unsigned long long total) {
    PtLayout L;
    L.off = 0;
    L.rect = L.off + align256((size_t)(N + 1) * sizeof(unsigned long long));
    L.w = L.rect + align256((size_t)N * sizeof(short4));
    L.err = L.w + align256((size_t)total * sizeof(float));
    L.bytes = L.err + 256;
    return L;
}

// The view of a fixed-view cache (creation view at this angle), checked.
int pt_view(pcas_solver s, double angle_rad, View* V) {
    pcas_cb cb = s->cb;
    cb.angle_rad = angle_rad;
    PCAS_TRY(make_view(&s->vol, &cb, s->prm.step_mm, V));
    if (cb.nu > 32767 || cb.nv > 32767)
        return fail(PCAS_ERR_INVALID_ARG, "fixed-view cache: detector sides must be at most 32767 pixels");
    return PCAS_OK;
}

// Footprint sizes of every voxel for this view, counted on the device into
// the solver's compacted-voxel scratch (free between solves; it holds at
// least N ints), then scanned: offsets into off (may be null) and the total
// into *d_total (device).
int pt_scan(pcas_solver s, const View& V, unsigned long long* off, unsigned long long* d_total, cudaStream_t st) {
    const Grid g = make_grid(&s->vol);
    const long N = (long)g.nx * g.ny * g.nz;
    unsigned int* area = reinterpret_cast<unsigned int*>(s->W.adj.act_idx);
    PCAS_LAUNCH(PCAS_K_INIT, st, launch_pt_count(V, g, area, st));
    PCAS_LAUNCH(PCAS_K_INIT, st, launch_pt_scan(area, N, off, d_total, st));
    return PCAS_OK;
}

}  // namespace

extern "C" {

size_t pcas_solver_fixed_view_bytes(pcas_solver s, double angle_rad, void* stream) {
    if (!s) return 0;
    View V;
    if (pt_view(s, angle_rad, &V) != PCAS_OK) return 0;
    cudaStream_t st = as_stream(stream);
    // the total lands in the gather's partials (free between solves)
    unsigned long long* d_total = reinterpret_cast<unsigned long long*>(s->W.part_adj);
    unsigned long long total = 0;
    if (pt_scan(s, V, nullptr, d_total, st) != PCAS_OK) return 0;
    if (cudaMemcpyAsync(&total, d_total, sizeof(total), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return 0;
    const long N = (long)s->vol.nx * s->vol.ny * s->vol.nz;
    return pt_layout(N, total).bytes;
}

int pcas_solver_fix_view(pcas_solver s, double angle_rad, void* cache, size_t cache_bytes, void* stream) {
    PCAS_TRY(check_ptr(s, "solver"));
    cudaStream_t st = as_stream(stream);
    PCAS_CUDA(cudaStreamSynchronize(st));         // no queued solve still reads the previous cache
    PCAS_CUDA(cudaStreamSynchronize(s->loc_stream));
    s->pt_on = 0;
    if (!cache) return PCAS_OK;                   // NULL: back to computing P^T in every gather
    if (((uintptr_t)cache & 255u) != 0) return fail(PCAS_ERR_INVALID_ARG, "fixed-view cache must be 256-byte aligned");
    if (!isfinite(angle_rad)) return fail(PCAS_ERR_INVALID_ARG, "angle_rad must be finite");
    View V;
    PCAS_TRY(pt_view(s, angle_rad, &V));
    const Grid g = make_grid(&s->vol);
    const long N = (long)g.nx * g.ny * g.nz;
    char* b = static_cast<char*>(cache);
    // the N + 1 offsets go to the start of the cache, the total to their end
    if (cache_bytes < pt_layout(N, 0).bytes)
        return fail(PCAS_ERR_INVALID_ARG, "fixed-view cache too small: %zu bytes", cache_bytes);
    unsigned long long* off = reinterpret_cast<unsigned long long*>(b);
    PCAS_TRY(pt_scan(s, V, off, off + N, st));
    unsigned long long total = 0;
    PCAS_CUDA(cudaMemcpyAsync(&total, off + N, sizeof(total), cudaMemcpyDeviceToHost, st));
    PCAS_CUDA(cudaStreamSynchronize(st));
    const PtLayout L = pt_layout(N, total);
    if (cache_bytes < L.bytes)
        return fail(PCAS_ERR_INVALID_ARG, "fixed-view cache too small: %zu < %zu bytes (pcas_solver_fixed_view_bytes)",
                    cache_bytes, L.bytes);
    short4* rect = reinterpret_cast<short4*>(b + L.rect);
    float* w = reinterpret_cast<float*>(b + L.w);
    int* err = reinterpret_cast<int*>(b + L.err);
    PCAS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    PCAS_LAUNCH(PCAS_K_INIT, st, launch_pt_build(V, g, off, rect, w, err, st));
    int herr = 0;
    PCAS_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    PCAS_CUDA(cudaStreamSynchronize(st));
    if (herr) return fail(PCAS_ERR_CUDA, "fixed-view cache: a footprint did not match its counted size");
    s->pt_rect = rect;
    s->pt_off = off;
    s->pt_w = w;
    s->pt_angle = angle_rad;
    s->pt_on = 1;
    return PCAS_OK;
}

int pcas_solver_solve(pcas_solver s, const float* y, double angle_rad, double off_u, double off_v,
                      const double* w_init, double* w_out, pcas_stats* stats, void* stream) {
    PCAS_TRY(check_ptr(s, "solver"));
    PCAS_TRY(check_ptr(w_init, "w_init"));
    cudaStream_t st = as_stream(stream);
    int slot;
    PCAS_TRY(solver_stage(s, angle_rad, off_u, off_v, w_init, 0, &slot, st));
    const size_t M = (size_t)s->cb.nu * s->cb.nv;
    if (y && y != s->y) PCAS_CUDA(cudaMemcpyAsync(s->y, y, M * sizeof(float), cudaMemcpyDeviceToDevice, st));
    PCAS_CUDA(cudaGraphLaunch(s->exec, st));
    PCAS_CUDA(cudaMemcpyAsync(s->h_state, s->W.st, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
    PCAS_CUDA(cudaEventRecord(s->ev[slot], st));
    PCAS_CUDA(cudaStreamSynchronize(st));
    s->seq_first = -1;                    // a solve in between ends a run
    {
        std::lock_guard<std::mutex> lk(g_prof_mutex);
        g_launches[PCAS_K_GRAPH] += s->h_state->launches;
    }
    return solver_collect(s, w_out, stats);
}

int pcas_solver_seq_begin(pcas_solver s, const double* lp_coef, int L, const double* c_ref, int loc_max_iter,
                          double loc_tol_mm, const double* w_hist, int n_hist, void* stream) {
    PCAS_TRY(check_ptr(s, "solver"));
    PCAS_TRY(check_ptr(lp_coef, "lp_coef"));
    PCAS_TRY(check_ptr(c_ref, "c_ref"));
    if (L < 1 || L > LP_MAX) return fail(PCAS_ERR_INVALID_ARG, "predictor order L must be in [1, %d]", (int)LP_MAX);
    if (n_hist < 0 || n_hist > LP_MAX || (n_hist > 0 && !w_hist))
        return fail(PCAS_ERR_INVALID_ARG, "n_hist must be in [0, %d] (w_hist non-NULL when > 0)", (int)LP_MAX);
    if (loc_max_iter < 1 || loc_max_iter > 100000 || !(loc_tol_mm > 0))
        return fail(PCAS_ERR_INVALID_ARG, "loc_max_iter must be in [1, 1e5] and loc_tol_mm > 0");
    PCAS_TRY(check_finite(lp_coef, s->K * L, "lp_coef"));
    PCAS_TRY(check_finite(c_ref, 3, "c_ref"));
    if (n_hist > 0) PCAS_TRY(check_finite(w_hist, s->K * n_hist, "w_hist"));
    cudaStream_t st = as_stream(stream);
    PCAS_CUDA(cudaStreamSynchronize(st));           // the previous run's copy of h_seq is done
    PCAS_CUDA(cudaStreamSynchronize(s->loc_stream));   // and its localisations (they read d_seq)
    SeqBlock& h = *s->h_seq;
    memset(&h, 0, sizeof(SeqBlock));
    for (int k = 0; k < s->K; k++)
        for (int l = 0; l < L; l++) h.lp[k * L + l] = lp_coef[k * L + l];
    for (int c = 0; c < 3; c++) h.c_ref[c] = c_ref[c];
    h.loc_tol = loc_tol_mm;
    h.loc_max_iter = loc_max_iter;
    h.o[0] = s->vol.ox; h.o[1] = s->vol.oy; h.o[2] = s->vol.oz;
    h.is[0] = 1.0 / s->vol.sx; h.is[1] = 1.0 / s->vol.sy; h.is[2] = 1.0 / s->vol.sz;
    h.L = L;
    h.n = n_hist;
    for (int l = 0; l < n_hist; l++)
        for (int k = 0; k < s->K; k++) h.hist[l][k] = w_hist[(size_t)l * s->K + k];
    PCAS_CUDA(cudaMemcpyAsync(s->d_seq, s->h_seq, sizeof(SeqBlock), cudaMemcpyHostToDevice, st));
    PCAS_CUDA(cudaStreamSynchronize(st));
    s->seq_first = s->next;
    return PCAS_OK;
}

int pcas_solver_seq_enqueue(pcas_solver s, const void* y, double angle_rad, const double* w_first,
                            long long* ticket, void* stream) {
    PCAS_TRY(check_ptr(s, "solver"));
    PCAS_TRY(check_ptr(ticket, "ticket"));
    if (s->seq_first < 0) return fail(PCAS_ERR_INVALID_ARG, "no run of projections: call pcas_solver_seq_begin");
    cudaStream_t st = as_stream(stream);
    int slot;
    PCAS_TRY(solver_stage(s, angle_rad, s->cb.off_u, s->cb.off_v, w_first, 1, &slot, st));
    const size_t bytes = (size_t)s->cb.nu * s->cb.nv * sizeof(float);
    if (y && y != s->y) {
        cudaPointerAttributes pa{};
        const bool host = cudaPointerGetAttributes(&pa, y) == cudaSuccess &&
                          (pa.type == cudaMemoryTypeHost || pa.type == cudaMemoryTypeUnregistered);
        cudaGetLastError();               // a failed query leaves no error behind
        if (host) {
            // the upload runs on the copy stream beside the projections
            // queued before this one; this solve waits only for its own image
            const int b = s->ynext;
            s->ynext ^= 1;
            PCAS_CUDA(cudaStreamWaitEvent(s->cp_stream, s->ev_used[b], 0));
            PCAS_CUDA(cudaMemcpyAsync(s->ystage[b], y, bytes, cudaMemcpyHostToDevice, s->cp_stream));
            PCAS_CUDA(cudaEventRecord(s->ev_cp[b], s->cp_stream));
            PCAS_CUDA(cudaStreamWaitEvent(st, s->ev_cp[b], 0));
            PCAS_CUDA(cudaMemcpyAsync(s->y, s->ystage[b], bytes, cudaMemcpyDeviceToDevice, st));
            PCAS_CUDA(cudaEventRecord(s->ev_used[b], st));
        } else {
            PCAS_CUDA(cudaMemcpyAsync(s->y, y, bytes, cudaMemcpyDefault, st));
        }
    }
    PCAS_CUDA(cudaGraphLaunch(s->exec, st));
    // the localisation and the result record on the solver's own stream, so
    // that the next projection's solve does not wait for them
    cudaStream_t ls = s->loc_stream;
    PCAS_CUDA(cudaEventRecord(s->ev_solved[slot], st));
    PCAS_CUDA(cudaStreamWaitEvent(ls, s->ev_solved[slot], 0));
    const Grid g = make_grid(&s->vol);
    SeqOut* d_res = s->d_out + slot;
    switch (s->dtype) {
        case DT_F32:
            k_seq_loc<float><<<1, 32, 0, ls>>>(s->d_seq, d_res, static_cast<const float*>(s->mean),
                                               static_cast<const float*>(s->U), s->K, g);
            break;
        case DT_BF16:
            k_seq_loc<__nv_bfloat16><<<1, 32, 0, ls>>>(s->d_seq, d_res, static_cast<const __nv_bfloat16*>(s->mean),
                                                       static_cast<const __nv_bfloat16*>(s->U), s->K, g);
            break;
        default:
            k_seq_loc<__half><<<1, 32, 0, ls>>>(s->d_seq, d_res, static_cast<const __half*>(s->mean),
                                                static_cast<const __half*>(s->U), s->K, g);
            break;
    }
    PCAS_CUDA(cudaGetLastError());
    PCAS_CUDA(cudaMemcpyAsync(&s->h_out[slot], d_res, sizeof(SeqOut), cudaMemcpyDeviceToHost, ls));
    PCAS_CUDA(cudaEventRecord(s->ev[slot], ls));
    s->slot_ticket[slot] = s->next - 1;
    s->slot_counted[slot] = false;
    *ticket = s->next - 1;
    return PCAS_OK;
}

int pcas_solver_seq_result(pcas_solver s, long long ticket, pcas_seq_result* out) {
    PCAS_TRY(check_ptr(s, "solver"));
    PCAS_TRY(check_ptr(out, "out"));
    if (ticket < 0) return fail(PCAS_ERR_INVALID_ARG, "ticket must be >= 0");
    const int slot = (int)(ticket % SEQ_RING);
    if (s->slot_ticket[slot] != ticket)
        return fail(PCAS_ERR_INVALID_ARG, "ticket %lld is not a pending or recent projection of a run", ticket);
    PCAS_CUDA(cudaEventSynchronize(s->ev[slot]));
    const SeqOut& h = s->h_out[slot];
    for (int k = 0; k < PCAS_KMAX; k++) out->w[k] = k < s->K ? h.w[k] : 0.0;
    for (int c = 0; c < 3; c++) out->c[c] = h.c[c];
    out->loc_converged = h.c[3] != 0.0;
    out->stats.iters = h.iters;
    out->stats.evals = h.evals;
    out->stats.status = h.phase == PH_SINGULAR ? PCAS_ERR_SINGULAR : PCAS_OK;
    out->stats.J0 = h.J0;
    out->stats.J = h.J;
    out->stats.a = h.a;
    out->stats.b = h.b;
    out->stats.mu_last = h.mu;
    if (!s->slot_counted[slot]) {
        s->slot_counted[slot] = true;
        std::lock_guard<std::mutex> lk(g_prof_mutex);
        g_launches[PCAS_K_GRAPH] += h.launches;
    }
    return out->stats.status;
}

int pcas_solver_destroy(pcas_solver s) {
    solver_free(s);
    return PCAS_OK;
}

int pcas_batch_create(pcas_batch* out, const pcas_solver* solvers, const float* const* y_src, int n,
                      void* stream) {
    PCAS_TRY(check_ptr(out, "out"));
    *out = nullptr;
    PCAS_TRY(check_ptr(solvers, "solvers"));
    if (n < 1 || n > 4096) return fail(PCAS_ERR_INVALID_ARG, "batch size must be in [1, 4096]");
    for (int i = 0; i < n; i++)
        if (!solvers[i]) return fail(PCAS_ERR_INVALID_ARG, "solver %d is NULL", i);
    (void)stream;
    pcas_batch b = new pcas_batch_s();
    b->solvers.assign(solvers, solvers + n);
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaGraphCreate(&b->graph, 0);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        if (b->graph) cudaGraphDestroy(b->graph);
        delete b;
        return fail(PCAS_ERR_CUDA, "batch set-up failed: %s", cudaGetErrorString(e));
    }
    int rc = PCAS_OK;
    for (int i = 0; i < n && rc == PCAS_OK; i++) rc = capture_solve(solvers[i], b->graph, cs, y_src ? y_src[i] : nullptr);
    cudaStreamDestroy(cs);
    if (rc == PCAS_OK) {
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) rc = fail(PCAS_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    if (rc != PCAS_OK) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        delete b;
        return rc;
    }
    *out = b;
    return PCAS_OK;
}

int pcas_batch_solve(pcas_batch b, const double* angle_rad, const double* w_init, double* w_out,
                     pcas_stats* stats, void* stream) {
    PCAS_TRY(check_ptr(b, "batch"));
    PCAS_TRY(check_ptr(angle_rad, "angle_rad"));
    PCAS_TRY(check_ptr(w_init, "w_init"));
    const int n = (int)b->solvers.size();
    cudaStream_t st = as_stream(stream);
    std::vector<int> slots(n);
    for (int i = 0; i < n; i++)
        PCAS_TRY(solver_stage(b->solvers[i], angle_rad[i], b->solvers[i]->cb.off_u, b->solvers[i]->cb.off_v,
                              w_init + (size_t)i * PCAS_KMAX, 0, &slots[i], st));
    PCAS_CUDA(cudaGraphLaunch(b->exec, st));
    for (int i = 0; i < n; i++) {
        pcas_solver si = b->solvers[i];
        PCAS_CUDA(cudaMemcpyAsync(si->h_state, si->W.st, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
        PCAS_CUDA(cudaEventRecord(si->ev[slots[i]], st));
        si->seq_first = -1;
    }
    PCAS_CUDA(cudaStreamSynchronize(st));
    int rc = PCAS_OK;
    long long launches = 0;
    for (int i = 0; i < n; i++) {
        launches += b->solvers[i]->h_state->launches;
        int r = solver_collect(b->solvers[i], w_out ? w_out + (size_t)i * PCAS_KMAX : nullptr,
                               stats ? stats + i : nullptr);
        if (stats && r != PCAS_OK) stats[i].status = r;
        if (r != PCAS_OK && rc == PCAS_OK) rc = r;
    }
    {
        std::lock_guard<std::mutex> lk(g_prof_mutex);
        g_launches[PCAS_K_GRAPH] += launches;
    }
    return rc;
}

int pcas_batch_destroy(pcas_batch b) {
    if (!b) return PCAS_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
    return PCAS_OK;
}

}  // extern "C"
