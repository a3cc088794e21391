// Device code of the FEWHA operator and the (augmented) PCG solver for sm_103a.
//
// Every step of the hot path is a "phase": a __device__ function that one CTA
// runs over the work items it owns (w = rank, rank + ncta, ...), where rank
// and ncta are the CTA's place in the group running this instance (the whole
// grid for one instance; a slice of it in the batched launch).
// The same phases run either as one kernel each (FEWHA_LAUNCH_PHASES) or back
// to back inside one persistent cooperative kernel separated by a bounded grid
// barrier (FEWHA_LAUNCH_PERSISTENT).  Reductions are deterministic: each CTA
// writes one partial per slot, and every consumer sums the partials of all
// CTAs in the same order.
//
// Phases (Ramlau & Stadler):
//   layer_idwt   W^{-1} per layer (Eq. fewha), fused with the direction update
//                of Algorithm 1/2 (p = z - mu p_m + beta p)
//   wfs          per guide star and pupil tile: P_g (Sec. 2, P^NGS / P^LGS),
//                Gamma (Sec. 2), C_eta^{-1}, Gamma^T, plus the data part of
//                (p, Mp) as a sum of weighted squared slopes
//   band_gather  P_g^T in gather form, per (layer, band of rows): the adjoint
//                wavefronts are staged in shared memory and contracted
//                separably (x then y), no atomics
//   layer_fdwt   W^{-T} per layer, fused with + alpha D p
//   axpy         c += alpha p, r -= alpha q and the inner products of
//                Algorithm 1/2 (z = J^{-1} r is never stored)
//   gram/init    projection of the warm start onto the recycled basis
//                (Algorithm 2 initial steps) with the k x k Gram matrix and
//                its Cholesky factor in FP64
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/fewha.h"

namespace fewha {

// 512 threads per CTA leave 128 registers per thread: with 1024 threads (64
// registers) the fused phases spilled ~300 bytes per thread to local memory.
constexpr int kThreads = 512;       // threads of every CTA
constexpr int kBandOutputs = 1024;  // layer nodes of one P^T work item (band of rows)
constexpr int kOutPT = (kBandOutputs + kThreads - 1) / kThreads;  // of them per thread
constexpr int kTabPT = 2;           // P^T weight-table entries staged per thread
constexpr int kMaxCtas = 1024;
constexpr int kK = FEWHA_MAX_K;
constexpr int kMaxT = 8;           // taps
constexpr int kAdjW = 8;           // most pupil nodes one layer node gathers from, per axis
constexpr int kSred = (4 + 2 * FEWHA_MAX_K) * 32;  // block_partials scratch (doubles)

// partial-sum slots (slot-major array part[slot * kMaxCtas + cta])
constexpr int kSlotE = 0;                       // parity p: + p*(4+2K): rz, zq, rp, rr, QTz[K], RP[K]
constexpr int kSlotEStride = 4 + 2 * kK;
constexpr int kSlotA = 2 * kSlotEStride;        // parity p: + 2p: pd, rz0
constexpr int kSlotB = kSlotA + 4;              // parity p: + p: ws
constexpr int kSlotR2 = kSlotB + 2;             // bb, rr
constexpr int kSlotGram = kSlotR2 + 2;          // K*K Gram entries (p_i, q_j), K entries (p_j, r)
constexpr int kSlotInit = kSlotGram + kK * kK + kK;  // K (q_j, z), rz, rr
constexpr int kSlots = kSlotInit + kK + 2;

struct Bar {
    unsigned int count, gen;  // arrivals; gen unused (kept for the layout)
};

// Device record of one solve (scalars shared between phases).
struct Record {
    int status, done, iters, chol_ok;
    double rz[FEWHA_MAX_ITER + 1];      // (r_k, z_k) after the projection of z_k
    double rinv[FEWHA_MAX_ITER + 1];    // 1 / rz[k]
    double alpha[FEWHA_MAX_ITER + 1];
    double L[FEWHA_MAX_K * FEWHA_MAX_K];  // Cholesky factor of the old basis' Gram matrix (row-major, kv x kv)
    double dinv[FEWHA_MAX_K];           // 1 / L_jj
    double rinv_pqm;                    // 1 / (p_m, q_m) of the newest recycled direction
    double bb;                          // ||b||^2 of this time step
    Bar bar;
};

template <typename T>
struct Geo {
    int G, L, ns, m;  // guide stars, layers, the geometry's (mirror's) subapertures and pupil nodes across
    long n;
    int lay_n[FEWHA_MAX_LAYERS], lay_J[FEWHA_MAX_LAYERS];
    long lay_off[FEWHA_MAX_LAYERS + 1];
    long ll_off[FEWHA_MAX_LAYERS + 1];  // (n_l/2)^2 blocks: level-1 approximation scratch
    T inv_delta[FEWHA_MAX_LAYERS];
    int n_taps;
    T h[kMaxT], g[kMaxT];
    int tile_y, tile_x;         // WFS tiles: tile_y x tile_x output nodes
    // sensors (guide star g): subapertures across, pupil nodes across, WFS
    // tiles per row of its pupil grid and tiles before it (WFS work items),
    // offsets of its P_g tables (fk, fw), adjoint wavefront (psi), slopes
    // and weights (wmask); m_max = the largest pupil grid
    int gs_ns[FEWHA_MAX_GS], gs_m[FEWHA_MAX_GS], gs_tiles_x[FEWHA_MAX_GS], gs_tile0[FEWHA_MAX_GS + 1];
    long gs_tab[FEWHA_MAX_GS], gs_psi[FEWHA_MAX_GS], gs_sl[FEWHA_MAX_GS], gs_mask[FEWHA_MAX_GS];
    int m_max;
    const int *fk, *alo, *ahi;  // interpolation tables
    const T *fw;
    const T *wmask;             // per sensor [n_g*n_g] weight on lit subapertures, 0 elsewhere
    const T *alpha_d;           // [n]
    const T *invJ;              // [n]
    int lay_lg[FEWHA_MAX_LAYERS];  // log2(n_l)
    int nbands;                 // P^T work items (layer, band of rows)
    const int *band_layer, *band_row0, *band_rows;  // [nbands]
    const int *band_ilo, *band_ihi;  // [G][nbands] pupil rows the band touches
    // guide stars of a band in groups whose pupil rows fit rows_chunk staged
    // rows: [G][nbands] end of the guide star's group, psi elements staged
    // before it within the group, and staged rows before it
    const int *band_gend, *band_gc, *band_gr;
    int rows_chunk;             // pupil rows staged per pass of band_gather
    int stage_tab;              // band_gather also stages its P^T weight tables in shared memory
    int pingpong;               // layer phases have a second n x n shared buffer
    // P_g^T weights per (g, l, axis, layer node k): pupil nodes adj_lo .. adj_lo +
    // adj_cnt - 1 with weights adj_w[..][0 .. adj_cnt), index ((g*L + l)*2 + axis)*FEWHA_MAX_GRID + k
    const int *adj_lo, *adj_cnt;
    const T *adj_w;             // [..][kAdjW]
    // y-contraction of a band as one list per (band, group, band row): staged
    // psi row and weight of every tap of every guide star of the group, in
    // guide-star then tap order; index ((w * G + g0) * ybr + r) (* ymax + t)
    const int *band_ycnt, *band_yrow;
    const T *band_yw;
    int ybr, ymax;
};

enum Mode { kApply = 0, kRhs = 1, kSolve = 2 };

template <typename T, typename S>
struct __align__(16) Args {
    Geo<T> geo;
    // operator buffers
    S *nodal;        // [n]  W^{-1} p (layer nodal values)
    S *psi;          // [G][m*m] Gamma^T C Gamma P_g (...) per guide star
    T *u;            // [n]  P^T psi (layer nodal adjoint)
    T *wq;           // [n]  W^{-T} u / delta (operator output before + alpha D p)
    T *ll;           // [sum (n_l/2)^2] level-1 approximation of each layer (split transforms)
    // working-precision (T) buffers of the residual replacement's operator
    // application: the nodal layers and adjoint wavefronts are stored in T
    // there even when S is narrower (== nodal / psi when S is T)
    T *nodal_t, *psi_t;
    const T *x;      // apply: input
    T *y;            // apply / rhs: output
    const S *slopes; // rhs / solve: measured slopes
    // solver
    T *c, *r, *b_prev;
    T *c_out;        // optional second destination of the solution (written at the end)
    T *P, *Q;        // [2][kcap][n]
    double *pq;      // [2][kcap]
    int *meta;
    int kcap;
    int max_iter, augmented, recycle_all;
    int true_res_every;  // N > 0: r <- b - M c after every N-th iteration (residual replacement)
    int rhs_in_state;    // b_prev = b and r_prev = r0 already: no right-hand-side phases
    double rtol;
    fewha_stats *stats;
    double *part;    // kSlots * kMaxCtas
    Record *rec;
    unsigned long long timeout_ns;
    int ncta;        // CTAs of the group running this instance
    int cta0;        // first CTA of that group (0 for a single instance)
    size_t smem_bytes;  // dynamic shared memory of every launch
    __device__ __forceinline__ int vrank() const { return (int)blockIdx.x - cta0; }
    unsigned long long *trace;  // optional phase trace [trace_cap][4]: start, last CTA done, barrier passed, tag
    int trace_cap;
    // derived per solve (host fills from nothing: phases read meta)
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
template <typename S>
struct Cv;
template <>
struct Cv<double> {
    __device__ static double ld(double v) { return v; }
    __device__ static double st(double v) { return v; }
};
template <>
struct Cv<float> {
    __device__ static float ld(float v) { return v; }
    __device__ static float st(float v) { return v; }
};
template <>
struct Cv<__nv_bfloat16> {
    __device__ static float ld(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static __nv_bfloat16 st(float v) { return __float2bfloat16_rn(v); }
};

// Loads of data another CTA of the same launch may have written: L2 only.
template <typename T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }
template <>
__device__ __forceinline__ __nv_bfloat16 ldcg<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    unsigned short u = __ldcg(reinterpret_cast<const unsigned short *>(p));
    return __ushort_as_bfloat16(u);
}
__device__ __forceinline__ double ldcgd(const double *p) { return __ldcg(p); }
__device__ __forceinline__ int ldcgi(const int *p) { return __ldcg(p); }

// 16-byte vector access (float4 / double2): W = 16 / sizeof(T) elements at a
// 16-byte aligned address.  vld_cg bypasses L1 (data written by another CTA
// of the same launch), vld_nc uses the read-only path (data constant for the
// launch).
template <typename T>
struct VW {
    static constexpr int W = 16 / sizeof(T);
};
__device__ __forceinline__ void vld_cg(const float *p, float (&x)[4])
{
    const float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
    x[0] = v.x, x[1] = v.y, x[2] = v.z, x[3] = v.w;
}
__device__ __forceinline__ void vld_cg(const double *p, double (&x)[2])
{
    const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
    x[0] = v.x, x[1] = v.y;
}
__device__ __forceinline__ void vld_nc(const float *p, float (&x)[4])
{
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    x[0] = v.x, x[1] = v.y, x[2] = v.z, x[3] = v.w;
}
__device__ __forceinline__ void vld_nc(const double *p, double (&x)[2])
{
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    x[0] = v.x, x[1] = v.y;
}
__device__ __forceinline__ void vld(const float *p, float (&x)[4])
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    x[0] = v.x, x[1] = v.y, x[2] = v.z, x[3] = v.w;
}
__device__ __forceinline__ void vld(const double *p, double (&x)[2])
{
    const double2 v = *reinterpret_cast<const double2 *>(p);
    x[0] = v.x, x[1] = v.y;
}
__device__ __forceinline__ void vst(float *p, const float (&x)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
}
__device__ __forceinline__ void vst(double *p, const double (&x)[2])
{
    *reinterpret_cast<double2 *>(p) = make_double2(x[0], x[1]);
}
__device__ __forceinline__ void vst(__nv_bfloat16 *p, const float (&x)[4])
{
    __nv_bfloat162 a = __floats2bfloat162_rn(x[0], x[1]), b = __floats2bfloat162_rn(x[2], x[3]);
    uint2 u;
    u.x = *reinterpret_cast<unsigned int *>(&a);
    u.y = *reinterpret_cast<unsigned int *>(&b);
    *reinterpret_cast<uint2 *>(p) = u;
}

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-thread / per-warp accumulation type: FP32 in the FP32 paths (FP64
// arithmetic runs at 1/64 of the FP32 rate on this part), FP64 in the FP64
// path.  Sums across warps and CTAs are always FP64.
template <typename T>
struct AccT {
    typedef float type;
};
template <>
struct AccT<double> {
    typedef double type;
};

template <typename A>
__device__ __forceinline__ A warp_sum_t(A v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of NV values per thread, written as partials of this CTA.
template <int NV, typename A>
__device__ void block_partials(A (&v)[NV], double *part, const int (&slot)[NV], double *sred, int cta)
// sred: shared scratch of NV * 32 doubles; cta: this CTA's rank in its group
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; i++) {
        A s = warp_sum_t(v[i]);
        if (lane == 0) sred[i * 32 + warp] = (double)s;
    }
    __syncthreads();
    if constexpr (NV <= kThreads / 32) {
        // one slot per warp at most: compile-time indices into slot[] (a
        // runtime index would place the caller's slot array in local memory)
#pragma unroll
        for (int i = 0; i < NV; i++) {
            if (i == warp) {
                double s = lane < nw ? sred[i * 32 + lane] : 0.0;
                s = warp_sum(s);
                if (lane == 0) part[(size_t)slot[i] * kMaxCtas + cta] = s;
            }
        }
    } else {
        for (int i = warp; i < NV; i += nw) {
            double s = lane < nw ? sred[i * 32 + lane] : 0.0;
            s = warp_sum(s);
            if (lane == 0) part[(size_t)slot[i] * kMaxCtas + cta] = s;
        }
    }
    __syncthreads();
}

// Sum over CTAs of `count` consecutive slots, into out[0..count) (shared).
__device__ inline void reduce_slots(const double *part, int ncta, int slot0, int count, double *out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = warp; s < count; s += nw) {
        const double *p = part + (size_t)(slot0 + s) * kMaxCtas;
        double acc = 0.0;
#pragma unroll 8
        for (int c = lane; c < ncta; c += 32) acc += __ldcg(p + c);
        acc = warp_sum(acc);
        if (lane == 0) out[s] = acc;
    }
    __syncthreads();
}

// Up to three contiguous slot ranges reduced in one round (one warp per slot).
struct SlotRange {
    int slot0, count;
    double *out;
};
__device__ inline void reduce_ranges(const double *part, int ncta, SlotRange r0, SlotRange r1 = {0, 0, nullptr},
                                     SlotRange r2 = {0, 0, nullptr})
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int total = r0.count + r1.count + r2.count;
    for (int s = warp; s < total; s += nw) {
        int slot;
        double *dst;
        if (s < r0.count) {
            slot = r0.slot0 + s;
            dst = r0.out + s;
        } else if (s < r0.count + r1.count) {
            slot = r1.slot0 + s - r0.count;
            dst = r1.out + s - r0.count;
        } else {
            slot = r2.slot0 + s - r0.count - r1.count;
            dst = r2.out + s - r0.count - r1.count;
        }
        const double *p = part + (size_t)slot * kMaxCtas;
        double v[8];
#pragma unroll
        for (int i = 0; i < 8; i++) v[i] = (lane + 32 * i < ncta) ? __ldcg(p + lane + 32 * i) : 0.0;
        double acc = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
        for (int c = lane + 256; c < ncta; c += 32) acc += __ldcg(p + c);
        acc = warp_sum(acc);
        if (lane == 0) *dst = acc;
    }
    __syncthreads();
}

// Sum over CTAs of `count` consecutive slots with the loads of every slot in
// one round: g lanes per slot (the largest power of two <= 32 with
// g * count <= blockDim.x), each summing every g-th partial, then a shuffle
// tree over the g lanes (fixed order).  For counts beyond the warps of a CTA.
__device__ inline void reduce_wide(const double *part, int ncta, int slot0, int count, double *out)
{
    int g = 32;
    while (g > 1 && g * count > (int)blockDim.x) g >>= 1;
    const int s = threadIdx.x / g, j = threadIdx.x - s * g;
    double acc = 0.0;
    if (s < count) {
        const double *p = part + (size_t)(slot0 + s) * kMaxCtas;
        double v[8];
#pragma unroll
        for (int i = 0; i < 8; i++) v[i] = (j + g * i < ncta) ? __ldcg(p + j + g * i) : 0.0;
        acc = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
#pragma unroll 4
        for (int c = j + 8 * g; c < ncta; c += g) acc += __ldcg(p + c);
    }
    for (int o = g >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (s < count && j == 0) out[s] = acc;
    __syncthreads();
}

// Warp-parallel Cholesky factorisation (right-looking) of the symmetrised
// k x k matrix G (row-major): L (row-major, k x k, lower) and dinv_j = 1/L_jj.
// Run by one full warp; returns false if not positive definite.
__device__ inline bool warp_cholesky(int k, const double *G, double *L, double *dinv)
{
    const int lane = threadIdx.x & 31;
    for (int e = lane; e < k * k; e += 32) {
        const int i = e / k, j = e - i * k;
        L[e] = i >= j ? 0.5 * (G[i * k + j] + G[j * k + i]) : 0.0;
    }
    __syncwarp();
    for (int j = 0; j < k; j++) {
        const double d = L[j * k + j];
        if (!(d > 0.0)) return false;
        const double r = rsqrt(d);
        __syncwarp();
        for (int i = j + 1 + lane; i < k; i += 32) L[i * k + j] *= r;
        if (lane == 0) {
            L[j * k + j] = d * r;
            dinv[j] = r;
        }
        __syncwarp();
        const int m = k - j - 1;
        for (int e = lane; e < m * m; e += 32) {
            const int i = j + 1 + e / m, t = j + 1 + e % m;
            if (t <= i) L[i * k + t] -= L[i * k + j] * L[t * k + j];
        }
        __syncwarp();
    }
    return true;
}

// Warp-parallel solve of L L^T x = rhs (factor from warp_cholesky); x may alias rhs.
__device__ inline void warp_chol_solve(int k, const double *L, const double *dinv, const double *rhs, double *x)
{
    const int lane = threadIdx.x & 31;
    double v = lane < k ? rhs[lane] : 0.0;
    for (int j = 0; j < k; j++) {  // forward: L y = rhs
        const double yj = __shfl_sync(0xffffffffu, v, j) * dinv[j];
        if (lane == j) v = yj;
        if (lane > j && lane < k) v -= L[lane * k + j] * yj;
    }
    for (int j = k - 1; j >= 0; j--) {  // backward: L^T x = y
        const double xj = __shfl_sync(0xffffffffu, v, j) * dinv[j];
        if (lane == j) v = xj;
        if (lane < j) v -= L[j * k + lane] * xj;
    }
    __syncwarp();
    if (lane < k) x[lane] = v;
    __syncwarp();
}

// Cholesky solve of the symmetrised k x k Gram matrix (row-major in Graw),
// one thread, factor in the k*k workspace A; false if not positive definite.
__device__ inline bool chol_solve(int k, const double *Graw, const double *rhs, double *x, double *A)
{
    for (int i = 0; i < k; i++)
        for (int j = 0; j < k; j++) A[i * k + j] = 0.5 * (Graw[i * k + j] + Graw[j * k + i]);
    for (int j = 0; j < k; j++) {
        double s = A[j * k + j];
        for (int t = 0; t < j; t++) s -= A[j * k + t] * A[j * k + t];
        if (!(s > 0.0)) return false;
        A[j * k + j] = sqrt(s);
        for (int i = j + 1; i < k; i++) {
            double v = A[i * k + j];
            for (int t = 0; t < j; t++) v -= A[i * k + t] * A[j * k + t];
            A[i * k + j] = v / A[j * k + j];
        }
    }
    for (int i = 0; i < k; i++) {
        double v = rhs[i];
        for (int t = 0; t < i; t++) v -= A[i * k + t] * x[t];
        x[i] = v / A[i * k + i];
    }
    for (int i = k - 1; i >= 0; i--) {
        double v = x[i];
        for (int t = i + 1; t < k; t++) v -= A[t * k + i] * x[t];
        x[i] = v / A[i * k + i];
    }
    return true;
}

// Error bit of the barrier counter: set together with the status, so that a
// CTA waiting at (or arriving at) a grid barrier sees the error in the word it
// polls anyway, without a second load.
constexpr unsigned int kBarErr = 0x80000000u;

__device__ __forceinline__ void set_status(Record *rec, int st)
{
    atomicCAS(&rec->status, 0, st);
    atomicOr(&rec->bar.count, kBarErr);
}

// Grid barrier with a time limit.  Returns false (and the CTA must return)
// when any CTA has recorded an error or the wait ran past timeout_ns.
// arrival: releases this CTA's writes and, for the last arriver, acquires
// everyone else's
__device__ __forceinline__ unsigned int atom_add_acq_rel_gpu(unsigned int *p, unsigned int v)
{
    unsigned int r;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "r"(v) : "memory");
    return r;
}
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p)
{
    unsigned int r;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(r) : "l"(p) : "memory");
    return r;
}
// Barrier over the nctas CTAs of a group, with a time limit.  Thread 0 arrives
// with an acquire-release add on a counter that only grows during a solve
// (after the block barrier, publishing the CTA's writes) and waits with
// acquire loads until the counter reaches the next multiple of nctas.  Returns
// false (and the CTA must return) when the counter's error bit is set (any CTA
// recorded an error) or the wait ran past timeout_ns.
// When this CTA passed its previous barrier (phase trace); trace_begin()
// stamps the start of the solve.
static __shared__ unsigned long long t_pass;

__device__ __forceinline__ void trace_begin(bool tracing)
{
    if (threadIdx.x == 0) t_pass = tracing ? gtimer() : 0ull;
}

__device__ inline bool grid_sync(Record *rec, unsigned long long timeout_ns, int nctas, int rank,
                                 unsigned long long *trace_slot = nullptr)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        if (trace_slot) {
            const unsigned long long now = gtimer();
            atomicMax(trace_slot + 1, now);
            if (t_pass) atomicMax(trace_slot, now - t_pass);
        }
        // the counter only grows within a solve (reset before every launch):
        // the barrier of this arrival completes when it reaches the next
        // multiple of nctas; an error anywhere sets its top bit
        const unsigned int prev = atom_add_acq_rel_gpu(&rec->bar.count, 1u);
        if (prev & kBarErr) {
            ok = 0;
        } else {
            const unsigned int target = (prev / (unsigned int)nctas + 1u) * (unsigned int)nctas;
            if (prev + 1u != target) {
                const unsigned long long t0 = gtimer();
                unsigned int polls = 0;
                for (;;) {
                    const unsigned int c = ld_acquire_gpu(&rec->bar.count);
                    if (c & kBarErr) {
                        ok = 0;
                        break;
                    }
                    if (c >= target) break;
                    if ((++polls & 7u) == 0u && gtimer() - t0 > timeout_ns) {  // time limit
                        set_status(rec, FEWHA_ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        if (trace_slot && rank == 0) trace_slot[2] = gtimer();
        t_pass = trace_slot ? gtimer() : 0ull;
    }
    __syncthreads();
    return ok != 0;
}

// ---------------------------------------------------------------------------
// Periodic orthonormal DWT passes in shared memory (Sec. 3, Eq. fewha)
//   analysis:  a_k = sum_t h_t x_{(2k+t) mod N},  d_k = sum_t g_t x_{(2k+t) mod N}
//   synthesis: x_{2m+e} = sum_u h_{e+2u} a_{(m-u) mod N/2} + g_{e+2u} d_{(m-u) mod N/2}
// The layer sits in shared memory row-major with pitch n + 1 (odd: one thread
// per row or per column is free of bank conflicts).  N is a power of two, so
// index reductions are bit masks.  The tap count L is a template parameter
// and the taps live in registers.  A thread computes kRun consecutive output
// pairs of one line from a register window (each input loaded once per run).
// ---------------------------------------------------------------------------
constexpr int kRun = 4;                          // output pairs per run

template <typename T, int L>
struct Taps {
    T h[L], g[L];
};

template <typename T, int L>
__device__ __forceinline__ Taps<T, L> load_taps(const Geo<T> &G)
{
    Taps<T, L> tp;
#pragma unroll
    for (int u = 0; u < L; u++) {
        tp.h[u] = G.h[u];
        tp.g[u] = G.g[u];
    }
    return tp;
}

// One run of `run` output pairs starting at pair m0 of the line at base
// (element stride es), into out[0 .. 2 kRun).
template <typename T, int L, bool SYNTH>
__device__ __forceinline__ void dwt_run(const T *base, int es, int N, int half, int run, int m0,
                                        const Taps<T, L> &tp, T (&out)[2 * kRun])
{
    constexpr int Lh = L / 2;
    if (SYNTH) {
        T wa[kRun + Lh - 1], wd[kRun + Lh - 1];  // a_{m0-Lh+1 .. m0+kRun-1}, same for d
#pragma unroll
        for (int i = 0; i < kRun + Lh - 1; i++) {
            if (i < run + Lh - 1) {
                const int k = (m0 - Lh + 1 + i) & (half - 1);
                wa[i] = base[k * es];
                wd[i] = base[(half + k) * es];
            } else {
                wa[i] = wd[i] = T(0);
            }
        }
#pragma unroll
        for (int q = 0; q < kRun; q++) {
            T x0 = 0, x1 = 0;
#pragma unroll
            for (int u = 0; u < Lh; u++) {
                const T a = wa[q + Lh - 1 - u], d = wd[q + Lh - 1 - u];
                x0 += tp.h[2 * u] * a + tp.g[2 * u] * d;
                x1 += tp.h[2 * u + 1] * a + tp.g[2 * u + 1] * d;
            }
            out[2 * q] = x0;
            out[2 * q + 1] = x1;
        }
    } else {
        T wx[2 * kRun + L - 2];  // x_{2 m0 .. 2 m0 + 2 kRun + L - 3}
#pragma unroll
        for (int i = 0; i < 2 * kRun + L - 2; i++)
            wx[i] = (i < 2 * run + L - 2) ? base[((2 * m0 + i) & (N - 1)) * es] : T(0);
#pragma unroll
        for (int q = 0; q < kRun; q++) {
            T a = 0, d = 0;
#pragma unroll
            for (int u = 0; u < L; u++) {
                a += tp.h[u] * wx[2 * q + u];
                d += tp.g[u] * wx[2 * q + u];
            }
            out[2 * q] = a;
            out[2 * q + 1] = d;
        }
    }
}

template <bool SYNTH, typename T>
__device__ __forceinline__ void dwt_store(T *base, int es, int half, int run, int m0, const T (&out)[2 * kRun])
{
#pragma unroll
    for (int q = 0; q < kRun; q++) {
        if (q < run) {
            const int p0 = SYNTH ? 2 * (m0 + q) : m0 + q;
            const int p1 = SYNTH ? 2 * (m0 + q) + 1 : half + m0 + q;
            base[p0 * es] = out[2 * q];
            base[p1 * es] = out[2 * q + 1];
        }
    }
}

// One pass over the top-left N x N block from src to dst (pitch P).  Thread
// idx takes line idx mod N and run idx / N: consecutive threads work on
// consecutive rows (ROWS) or columns.  FP32: dst is the ping-pong buffer.
// FP64 (a 128 x 129 layer fills 132 KB): in place (src == dst), one warp per
// line at a time.
template <typename T, int L, bool ROWS, bool SYNTH>
__device__ void dwt_pass(const T *src, T *dst, int P, int lgN, const Geo<T> &G)
{
    // taps read here (shared memory), live only during the pass
    const Taps<T, L> tp = load_taps<T, L>(G);
    const int N = 1 << lgN, half = N >> 1;
    const int run = half < kRun ? half : kRun;       // pairs per run
    const int total = N * (half / run);              // runs in the pass
    const int es = ROWS ? 1 : P;                     // element stride along a line
    const int ls = ROWS ? P : 1;                     // stride between lines
    if constexpr (sizeof(T) == 4) {
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int line = idx & (N - 1), m0 = (idx >> lgN) * run;
            T out[2 * kRun];
            dwt_run<T, L, SYNTH>(src + line * ls, es, N, half, run, m0, tp, out);
            dwt_store<SYNTH>(dst + line * ls, es, half, run, m0, out);
        }
        __syncthreads();
    } else {
        // in place (FP64): a line's outputs overwrite only that line, so the
        // lanes of one warp read the whole line into registers, synchronise
        // and write it back; a warp takes 32 / (runs per line) lines at once
        // (N <= FEWHA_MAX_GRID = 128: at most 16 runs of 4 pairs per line)
        const int nr = half / run, lpw = 32 / nr;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        const int sub = lane / nr, m0 = (lane - sub * nr) * run;
        for (int line0 = warp * lpw; line0 < N; line0 += nw * lpw) {
            const int line = line0 + sub;
            const bool act = line < N;
            T out[2 * kRun];
            if (act) dwt_run<T, L, SYNTH>(src + line * ls, es, N, half, run, m0, tp, out);
            __syncwarp();
            if (act) dwt_store<SYNTH>(dst + line * ls, es, half, run, m0, out);
        }
        __syncthreads();
    }
}

// Multi-level transforms of an n x n layer in buf (pitch n + 1); tmp is a
// second buffer (FP32 ping-pong: both passes of a level return to buf) or buf.
template <typename T, int L>
__device__ void idwt2_L(T *buf, T *tmp, int lgn, int J, const Geo<T> &G)
{
    const int P = (1 << lgn) + 1;
    for (int t = J - 1; t >= 0; t--) {
        dwt_pass<T, L, false, true>(buf, tmp, P, lgn - t, G);
        dwt_pass<T, L, true, true>(tmp, buf, P, lgn - t, G);
    }
}

template <typename T, int L>
__device__ void fdwt2_L(T *buf, T *tmp, int lgn, int J, const Geo<T> &G)
{
    const int P = (1 << lgn) + 1;
    for (int t = 0; t < J; t++) {
        dwt_pass<T, L, true, false>(buf, tmp, P, lgn - t, G);
        dwt_pass<T, L, false, false>(tmp, buf, P, lgn - t, G);
    }
}

// Daubechies-1..4 (2..8 taps)
template <typename T>
__device__ void idwt2(T *buf, T *tmp, int lgn, int J, const Geo<T> &G)
{
    switch (G.n_taps) {
    case 2: idwt2_L<T, 2>(buf, tmp, lgn, J, G); break;
    case 4: idwt2_L<T, 4>(buf, tmp, lgn, J, G); break;
    case 6: idwt2_L<T, 6>(buf, tmp, lgn, J, G); break;
    default: idwt2_L<T, 8>(buf, tmp, lgn, J, G); break;
    }
}

template <typename T>
__device__ void fdwt2(T *buf, T *tmp, int lgn, int J, const Geo<T> &G)
{
    switch (G.n_taps) {
    case 2: fdwt2_L<T, 2>(buf, tmp, lgn, J, G); break;
    case 4: fdwt2_L<T, 4>(buf, tmp, lgn, J, G); break;
    case 6: fdwt2_L<T, 6>(buf, tmp, lgn, J, G); break;
    default: fdwt2_L<T, 8>(buf, tmp, lgn, J, G); break;
    }
}

// Layer element e (row-major, n columns) <-> shared-memory index (pitch n + 1).
__device__ __forceinline__ int spad(int e, int lgn) { return e + (e >> lgn); }

template <typename T, typename S, class Load>
__device__ void layer_idwt(const Args<T, S> &A, T *buf, Load load)
{
    constexpr int W = VW<T>::W;
    const Geo<T> &G = A.geo;
    for (int l = A.vrank(); l < G.L; l += A.ncta) {
        const int n = G.lay_n[l], lgn = G.lay_lg[l], nv = n * n / W;
        const long off = G.lay_off[l];
#pragma unroll 2
        for (int v = threadIdx.x; v < nv; v += blockDim.x) {
            T x[W];
            load(off + (long)v * W, x);
            const int s0 = spad(v * W, lgn);
#pragma unroll
            for (int i = 0; i < W; i++) buf[s0 + i] = x[i];
        }
        __syncthreads();
        idwt2<T>(buf, G.pingpong ? buf + n * (n + 1) : buf, lgn, G.lay_J[l], G);
        const T sc = G.inv_delta[l];
        for (int v = threadIdx.x; v < nv; v += blockDim.x) {
            T x[W];
            const int s0 = spad(v * W, lgn);
#pragma unroll
            for (int i = 0; i < W; i++) x[i] = buf[s0 + i] * sc;
            vst(A.nodal + off + (long)v * W, x);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// WFS phase: per guide star g and tile of tile x tile pupil nodes.
//   OP mode : phi = P_g nodal at the tile's nodes plus a one-node halo,
//             slopes = Gamma phi (Sec. 2), weighted by C_eta^{-1};
//             returns sum of w s^2 over the tile's own subapertures
//   RHS mode: weighted slopes from the measured slopes
//   both    : psi_g = Gamma^T (weighted slopes) on the tile's nodes.
// ---------------------------------------------------------------------------
template <typename T, typename S, bool RHS>
__device__ __forceinline__ typename AccT<T>::type wfs_phase(const Args<T, S> &A, T *sm)
{
    typedef typename AccT<T>::type Acc;
    const Geo<T> &G = A.geo;
    const int TY = G.tile_y, TX = G.tile_x, HY = TY + 2, HX = TX + 2, SY = TY + 1, SX = TX + 1;
    const int total = G.gs_tile0[G.G];
    T *phi = sm;                          // [HY*HX] sum over layers (OP)
    T *sx = sm + (size_t)G.L * HY * HX;   // [SY*SX]
    T *sy = sx + SY * SX;
    Acc ws = 0;
    for (int w = A.vrank(); w < total; w += A.ncta) {
        int g = 0;
        while (w >= G.gs_tile0[g + 1]) g++;  // sensor of this work item
        const int m = G.gs_m[g], ns = G.gs_ns[g], tt = w - G.gs_tile0[g];
        const int i0 = (tt / G.gs_tiles_x[g]) * TY, j0 = (tt % G.gs_tiles_x[g]) * TX;
        if (!RHS) {
            // phi at each halo node: the sum over layers of the bilinear value of
            // the layer at the node's projection (layer after layer, from 0),
            // with the loads of kLC layers in flight at once
            constexpr int kLC = 9;
            for (int loc = threadIdx.x; loc < HY * HX; loc += blockDim.x) {
                const int i = i0 - 1 + loc / HX, j = j0 - 1 + loc % HX;
                T sum = 0;
                if (i >= 0 && i < m && j >= 0 && j < m) {
                    for (int l0 = 0; l0 < G.L; l0 += kLC) {
                        T v[kLC];
#pragma unroll
                        for (int u = 0; u < kLC; u++) {
                            const int l = l0 + u;
                            v[u] = 0;
                            if (l < G.L) {
                                const long bx = G.gs_tab[g] + (long)(l * 2 + 0) * m;
                                const long by = G.gs_tab[g] + (long)(l * 2 + 1) * m;
                                const int kx = __ldg(G.fk + bx + j), ky = __ldg(G.fk + by + i);
                                const T wx = __ldg(G.fw + bx + j), wy = __ldg(G.fw + by + i);
                                const int n = G.lay_n[l];
                                const S *Lp = A.nodal + G.lay_off[l] + (long)ky * n + kx;
                                const T v00 = Cv<S>::ld(ldcg(Lp)), v01 = Cv<S>::ld(ldcg(Lp + 1));
                                const T v10 = Cv<S>::ld(ldcg(Lp + n)), v11 = Cv<S>::ld(ldcg(Lp + n + 1));
                                v[u] = (T(1) - wy) * ((T(1) - wx) * v00 + wx * v01) + wy * ((T(1) - wx) * v10 + wx * v11);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < kLC; u++) sum += v[u];
                    }
                }
                phi[loc] = sum;
            }
            __syncthreads();
        }
        // weighted slopes of subapertures (i0-1 .. i0+TY-1) x (j0-1 .. j0+TX-1)
        for (int e = threadIdx.x; e < SY * SX; e += blockDim.x) {
            const int a = e / SX, b = e - a * SX;
            const int i = i0 - 1 + a, j = j0 - 1 + b;
            T vx = 0, vy = 0;
            if (i >= 0 && i < ns && j >= 0 && j < ns) {
                const T wgt = __ldg(G.wmask + G.gs_mask[g] + i * ns + j);
                if (RHS) {
                    const S *sg = A.slopes + G.gs_sl[g];
                    vx = wgt * Cv<S>::ld(sg[i * ns + j]);
                    vy = wgt * Cv<S>::ld(sg[ns * ns + i * ns + j]);
                } else {
                    const T p00 = phi[a * HX + b], p01 = phi[a * HX + b + 1];
                    const T p10 = phi[(a + 1) * HX + b], p11 = phi[(a + 1) * HX + b + 1];
                    const T gx = T(0.5) * ((p01 - p00) + (p11 - p10));
                    const T gy = T(0.5) * ((p10 - p00) + (p11 - p01));
                    vx = wgt * gx;
                    vy = wgt * gy;
                    if (a >= 1 && b >= 1) ws += (Acc)vx * (Acc)gx + (Acc)vy * (Acc)gy;
                }
            }
            sx[e] = vx;
            sy[e] = vy;
        }
        __syncthreads();
        // Gamma^T on the tile's own nodes
        for (int e = threadIdx.x; e < TY * TX; e += blockDim.x) {
            const int a = e / TX + 1, b = e % TX + 1;  // subaperture-local (i, j) of node (i0+a-1, j0+b-1)
            const int i = i0 + a - 1, j = j0 + b - 1;
            if (i < m && j < m) {
                const T v = T(0.5) * (sx[a * SX + b - 1] - sx[a * SX + b] + sx[(a - 1) * SX + b - 1] -
                                      sx[(a - 1) * SX + b] + sy[(a - 1) * SX + b] - sy[a * SX + b] +
                                      sy[(a - 1) * SX + b - 1] - sy[a * SX + b - 1]);
                A.psi[G.gs_psi[g] + i * m + j] = Cv<S>::st(v);
            }
        }
        __syncthreads();
    }
    return ws;
}

// ---------------------------------------------------------------------------
// P^T phase: u = sum_g P_g^T psi_g, gather form, one work item per (layer l,
// band of layer rows [a0, a0+BR)).  P_g restricted to layer l is separable,
// Wy (x) Wx, so per guide star
//     T[i][b] = sum_j Wx[j][b] psi_g[i][j]     (pupil rows i the band touches)
//     u[a][b] += sum_i Wy[i][a] T[i][b]
// with psi rows staged in shared memory in chunks of rows_chunk rows.
// Thread (a - a0, b) owns output u[a][b]; no atomics, fixed summation order.
// ---------------------------------------------------------------------------
// Header of a P^T work item for guide star threadIdx.x (< G): pupil rows and
// group of the band, loaded ahead of time by band_header().
struct BandHdr {
    int ilo, ihi, gend, gc, gr;
};

template <typename T, typename S>
__device__ __forceinline__ BandHdr band_header(const Args<T, S> &A, int w)
{
    BandHdr h = {0, 0, 0, 0, 0};
    const Geo<T> &G = A.geo;
    if (threadIdx.x < G.G && w < G.nbands) {
        const int i = threadIdx.x * G.nbands + w;
        h.ilo = __ldg(G.band_ilo + i);
        h.ihi = __ldg(G.band_ihi + i);
        h.gend = __ldg(G.band_gend + i);
        h.gc = __ldg(G.band_gc + i);
        h.gr = __ldg(G.band_gr + i);
    }
    return h;
}

// pre: the header of the CTA's first work item (w = A.vrank()), when the
// caller loaded it before other work to hide its latency
template <typename T, typename S>
__device__ __forceinline__ void band_gather(const Args<T, S> &A, T *sm, const BandHdr *pre = nullptr)
{
    const Geo<T> &G = A.geo;
    const int RC = G.rows_chunk, NB = G.nbands;
    __shared__ int s_cum[FEWHA_MAX_GS + 1], s_base[FEWHA_MAX_GS + 1];
    __shared__ int s_ilo[FEWHA_MAX_GS], s_ihi[FEWHA_MAX_GS], s_gend[FEWHA_MAX_GS], s_gc[FEWHA_MAX_GS];
    __shared__ int s_gr[FEWHA_MAX_GS];
    __shared__ long s_off[FEWHA_MAX_GS];  // psi element = s_off[q] + staged index
    for (int w = A.vrank(); w < NB; w += A.ncta) {
        const int l = __ldg(G.band_layer + w), a0 = __ldg(G.band_row0 + w), BR = __ldg(G.band_rows + w);
        const int n = G.lay_n[l], lgn = G.lay_lg[l], nout = BR << lgn;
        // owned outputs o = threadIdx.x + j blockDim.x: layer node (a0 + (o >> lgn), o & (n - 1))
        T acc[kOutPT];
#pragma unroll
        for (int j = 0; j < kOutPT; j++) acc[j] = 0;
        // staged psi rows (guide star q's rows of its gs_m[q] nodes, one after
        // the other: at most RC rows of m_max) and their x-contraction [RC][n]
        T *ps = sm;
        T *Tb = sm + RC * G.m_max;
        // pupil rows [ilo, ihi) of every guide star for this band and its
        // group (precomputed on the host), one load each in parallel
        if (threadIdx.x < G.G) {
            const BandHdr h = (pre && w == A.vrank()) ? *pre : band_header(A, w);
            s_ilo[threadIdx.x] = h.ilo;
            s_ihi[threadIdx.x] = h.ihi;
            s_gend[threadIdx.x] = h.gend;
            s_gc[threadIdx.x] = h.gc;
            s_gr[threadIdx.x] = h.gr;
        }
        __syncthreads();
        // guide stars in groups whose pupil rows fit the RC staged rows
        for (int g0 = 0, g1; g0 < G.G; g0 = g1) {
            g1 = s_gend[g0];
            const int ng = g1 - g0;
            // stage psi rows of the group's guide stars, flattened so that each
            // thread has all of its loads in flight at once (one latency round);
            // the staging offsets of the group are filled in parallel
            if (threadIdx.x <= ng) {
                const int q = threadIdx.x, g = g0 + q;
                const int rl = s_ihi[g1 - 1] - s_ilo[g1 - 1];  // rows of the group's last guide star
                const int c = q < ng ? s_gc[g] : s_gc[g1 - 1] + rl * G.gs_m[g1 - 1];
                s_cum[q] = c;
                s_base[q] = q < ng ? s_gr[g] : s_gr[g1 - 1] + rl;
                if (q < ng) s_off[q] = G.gs_psi[g] + (long)s_ilo[g] * G.gs_m[g] - c;
            }
            __syncthreads();
            const int nxt = ng << lgn;
            // x weight tables of the group (per guide star and layer column),
            // loaded in the same latency round as the psi rows
            T *xw = Tb + RC * n;                          // [kAdjW][ng * n] (tap-major: no bank conflicts)
            int *xlo = reinterpret_cast<int *>(xw + (size_t)nxt * kAdjW), *xct = xlo + nxt;
            const bool tab = G.stage_tab != 0;
            // table entries tt = threadIdx.x + j blockDim.x (nxt <= kTabPT blockDim.x)
            int t_lo[kTabPT], t_ct[kTabPT];
            T t_w[kTabPT][kAdjW];
#pragma unroll
            for (int j = 0; j < kTabPT; j++) {
                const int tt = threadIdx.x + j * blockDim.x;
                t_lo[j] = t_ct[j] = 0;
                if (tab && tt < nxt) {
                    const int q = tt >> lgn, bcol = tt & (n - 1);
                    const int idx = ((g0 + q) * G.L + l) * 2 * FEWHA_MAX_GRID + bcol;
                    t_lo[j] = __ldg(G.adj_lo + idx);
                    t_ct[j] = __ldg(G.adj_cnt + idx);
#pragma unroll
                    for (int c = 0; c < kAdjW; c++) t_w[j][c] = __ldg(G.adj_w + (size_t)idx * kAdjW + c);
                }
            }
            {
                const int total = s_cum[ng];
                constexpr int U = 8;
                int q = 0;  // guide star of the staged index t (t only grows)
                for (int t0 = threadIdx.x; t0 < total; t0 += U * blockDim.x) {
                    S v[U];
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const int t = t0 + u * blockDim.x;
                        if (t < total) {
                            while (t >= s_cum[q + 1]) q++;
                            v[u] = ldcg(A.psi + s_off[q] + t);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const int t = t0 + u * blockDim.x;
                        if (t < total) ps[t] = Cv<S>::ld(v[u]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < kTabPT; j++) {
                const int tt = threadIdx.x + j * blockDim.x;
                if (tab && tt < nxt) {
                    xlo[tt] = t_lo[j];
                    xct[tt] = t_ct[j];
#pragma unroll
                    for (int c = 0; c < kAdjW; c++) xw[(size_t)c * nxt + tt] = t_w[j][c];
                }
            }
            __syncthreads();
            // x-contraction: Tb[i][b] = sum_j Wx[j][b] psi[i][j]
            {
                const int total = s_base[ng];  // staged rows
                int q = 0;                     // guide star of the staged row (rows only grow)
                if (tab && (int)blockDim.x % n == 0 && (blockDim.x & (blockDim.x - 1)) == 0) {
                    // each thread keeps one column b and the rows r0 + k rstep
                    // (rstep = blockDim.x / n, a power of two: rows congruent to
                    // r0 modulo rstep, found with a mask);
                    // guide star after guide star, its weights in registers and
                    // the taps unrolled up to the warp's largest count
                    const int bcol = threadIdx.x & (n - 1), r0 = threadIdx.x >> lgn, rstep = blockDim.x >> lgn;
                    for (q = 0; q < ng; q++) {
                        const int ti = (q << lgn) + bcol;
                        const int jlo = xlo[ti], cnt = xct[ti];
                        const int cmax = __reduce_max_sync(0xffffffffu, (unsigned)cnt);
                        T wr[kAdjW];
#pragma unroll
                        for (int c = 0; c < kAdjW; c++) wr[c] = c < cnt ? xw[(size_t)c * nxt + ti] : T(0);
                        const int rb = s_base[q], re = s_base[q + 1], mq = G.gs_m[g0 + q];
                        for (int row = rb + ((r0 - rb) & (rstep - 1)); row < re; row += rstep) {
                            const T *rowp = ps + s_cum[q] + (row - rb) * mq + jlo;
                            T v = 0;
#pragma unroll
                            for (int c = 0; c < kAdjW; c++)
                                if (c < cmax && c < cnt) v += wr[c] * rowp[c];
                            Tb[(row << lgn) + bcol] = v;
                        }
                    }
                } else {
                    for (int e = threadIdx.x; e < (total << lgn); e += blockDim.x) {
                        const int row = e >> lgn, bcol = e & (n - 1);
                        while (row >= s_base[q + 1]) q++;
                        int jlo, cnt, ws;
                        const T *wt;
                        if (tab) {
                            const int ti = (q << lgn) + bcol;
                            jlo = xlo[ti];
                            cnt = xct[ti];
                            wt = xw + ti;
                            ws = nxt;
                        } else {
                            const int tx = ((g0 + q) * G.L + l) * 2 * FEWHA_MAX_GRID + bcol;
                            jlo = __ldg(G.adj_lo + tx);
                            cnt = __ldg(G.adj_cnt + tx);
                            wt = G.adj_w + (size_t)tx * kAdjW;
                            ws = 1;
                        }
                        const T *rowp = ps + s_cum[q] + (row - s_base[q]) * G.gs_m[g0 + q] + jlo;
                        T v = 0;
                        for (int c = 0; c < cnt; c++) v += wt[c * ws] * rowp[c];  // cnt <= kAdjW
                        Tb[(row << lgn) + bcol] = v;
                    }
                }
            }
            __syncthreads();
            // y-contraction into the owned outputs: the band row's tap list of
            // this group (staged row, weight), the same for the lanes of a warp
#pragma unroll
            for (int j = 0; j < kOutPT; j++) {
                const int o = threadIdx.x + j * blockDim.x;
                if (o < nout) {
                    const size_t e = ((size_t)w * G.G + g0) * G.ybr + (o >> lgn);
                    const int cnt = __ldg(G.band_ycnt + e);
                    const int *yr = G.band_yrow + e * G.ymax;
                    const T *yv = G.band_yw + e * G.ymax;
                    const T *col = Tb + (o & (n - 1));
                    for (int t = 0; t < cnt; t++) acc[j] += __ldg(yv + t) * col[__ldg(yr + t) << lgn];
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < kOutPT; j++) {
            const int o = threadIdx.x + j * blockDim.x;
            if (o < nout) A.u[G.lay_off[l] + ((long)(a0 + (o >> lgn)) << lgn) + (o & (n - 1))] = acc[j];
        }
    }
}

// ---------------------------------------------------------------------------
// Layer phase 2: W u / delta_l per layer; `store(e, value)` consumes each
// coefficient (u was written by band_gather in another CTA: L2 loads).
// ---------------------------------------------------------------------------
template <typename T, typename S, class Store>
__device__ void layer_fdwt(const Args<T, S> &A, T *buf, Store store)
{
    constexpr int W = VW<T>::W;
    const Geo<T> &G = A.geo;
    for (int l = A.vrank(); l < G.L; l += A.ncta) {
        const int n = G.lay_n[l], lgn = G.lay_lg[l], nv = n * n / W;
        const long off = G.lay_off[l];
#pragma unroll 4
        for (int v = threadIdx.x; v < nv; v += blockDim.x) {
            T x[W];
            vld_cg(A.u + off + (long)v * W, x);
            const int s0 = spad(v * W, lgn);
#pragma unroll
            for (int i = 0; i < W; i++) buf[s0 + i] = x[i];
        }
        __syncthreads();
        fdwt2<T>(buf, G.pingpong ? buf + n * (n + 1) : buf, lgn, G.lay_J[l], G);
        const T sc = G.inv_delta[l];
#pragma unroll 2
        for (int v = threadIdx.x; v < nv; v += blockDim.x) {
            T x[W];
            const int s0 = spad(v * W, lgn);
#pragma unroll
            for (int i = 0; i < W; i++) x[i] = buf[s0 + i] * sc;
            store(off + (long)v * W, x);
        }
        __syncthreads();
    }
}

// Element range of this CTA for vector phases, aligned to W elements.
__device__ __forceinline__ void cta_range_vec(long n, int W, int rank, int nctas, long &lo, long &hi)
{
    long nv = n / W;
    long chunk = (nv + nctas - 1) / nctas;
    lo = (long)rank * chunk * W;
    hi = lo + chunk * W < n ? lo + chunk * W : n;
}

// Element range of this CTA for vector phases.
__device__ __forceinline__ void cta_range(long n, int rank, int nctas, long &lo, long &hi)
{
    long chunk = (n + nctas - 1) / nctas;
    lo = (long)rank * chunk;
    hi = lo + chunk < n ? lo + chunk : n;
}

}  // namespace fewha
