// Device code of the FEWHA operator and the (augmented) PCG solver for sm_103a.
//
// Every step of the hot path is a "phase": a __device__ function that one CTA
// runs over the work items it owns (w = blockIdx.x, blockIdx.x + gridDim.x, ...).
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

constexpr int kThreads = 1024;     // threads of every CTA
constexpr int kPairs = 8;          // DWT output pairs per thread: 128 * 64 / 1024
constexpr int kMaxCtas = 1024;
constexpr int kK = FEWHA_MAX_K;
constexpr int kMaxT = 8;           // taps

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
    unsigned int count, gen;
};

// Device record of one solve (scalars shared between phases).
struct Record {
    int status, done, iters, frame_bank;
    double rz[FEWHA_MAX_ITER + 1];
    double alpha[FEWHA_MAX_ITER + 1];
    Bar bar;
};

template <typename T>
struct Geo {
    int G, L, ns, m;
    long n;
    int lay_n[FEWHA_MAX_LAYERS], lay_J[FEWHA_MAX_LAYERS];
    long lay_off[FEWHA_MAX_LAYERS + 1];
    T inv_delta[FEWHA_MAX_LAYERS];
    int n_taps;
    T h[kMaxT], g[kMaxT];
    int tile, tiles_x;          // WFS tiles: tile x tile output nodes, tiles_x per axis
    const int *fk, *alo, *ahi;  // interpolation tables
    const T *fw;
    const T *wmask;             // [G][ns*ns] weight on lit subapertures, 0 elsewhere
    const T *alpha_d;           // [n]
    const T *invJ;              // [n]
    int lay_lg[FEWHA_MAX_LAYERS];  // log2(n_l)
    int nbands;                 // P^T work items (layer, band of rows)
    const int *band_layer, *band_row0, *band_rows;  // [nbands]
    const int *band_ilo, *band_ihi;  // [G][nbands] pupil rows the band touches
    int rows_chunk;             // pupil rows staged per pass of band_gather
};

enum Mode { kApply = 0, kRhs = 1, kSolve = 2 };

template <typename T, typename S>
struct Args {
    Geo<T> geo;
    // operator buffers
    S *nodal;        // [n]  W^{-1} p (layer nodal values)
    S *psi;          // [G][m*m] Gamma^T C Gamma P_g (...) per guide star
    T *u;            // [n]  P^T psi (layer nodal adjoint)
    const T *x;      // apply: input
    T *y;            // apply / rhs: output
    const S *slopes; // rhs / solve: measured slopes
    // solver
    T *c, *r, *b_prev;
    T *P, *Q;        // [2][kcap][n]
    double *pq;      // [2][kcap]
    int *meta;
    int kcap;
    int max_iter, augmented, recycle_all;
    double rtol;
    fewha_stats *stats;
    double *part;    // kSlots * kMaxCtas
    Record *rec;
    unsigned long long timeout_ns;
    int ncta;        // CTAs that wrote partials (the solver grid)
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
__device__ void block_partials(A (&v)[NV], double *part, const int (&slot)[NV], double *sred)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; i++) {
        A s = warp_sum_t(v[i]);
        if (lane == 0) sred[i * 32 + warp] = (double)s;
    }
    __syncthreads();
    if (warp < NV) {
        double s = lane < nw ? sred[warp * 32 + lane] : 0.0;
        s = warp_sum(s);
        if (lane == 0) part[(size_t)slot[warp] * kMaxCtas + blockIdx.x] = s;
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
        for (int c = lane; c < ncta; c += 32) acc += __ldcg(p + c);
        acc = warp_sum(acc);
        if (lane == 0) out[s] = acc;
    }
    __syncthreads();
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

__device__ __forceinline__ void set_status(Record *rec, int st)
{
    atomicCAS(&rec->status, 0, st);
}

// Grid barrier with a time limit.  Returns false (and the CTA must return)
// when any CTA has recorded an error or the wait ran past timeout_ns.
__device__ inline bool grid_sync(Record *rec, unsigned long long timeout_ns)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned int *vgen = &rec->bar.gen;
        volatile int *vst = &rec->status;
        unsigned int g = *vgen;
        __threadfence();
        unsigned int prev = atomicAdd(&rec->bar.count, 1u);
        if (prev == gridDim.x - 1) {
            atomicExch(&rec->bar.count, 0u);
            __threadfence();
            atomicAdd(&rec->bar.gen, 1u);
        } else {
            unsigned long long t0 = gtimer();
            while (*vgen == g) {
                if (*vst != 0) {
                    ok = 0;
                    break;
                }
                if (gtimer() - t0 > timeout_ns) {
                    set_status(rec, FEWHA_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        if (*vst != 0) ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

// ---------------------------------------------------------------------------
// Periodic orthonormal DWT passes in shared memory (Sec. 3, Eq. fewha)
//   analysis:  a_k = sum_t h_t x_{(2k+t) mod N},  d_k = sum_t g_t x_{(2k+t) mod N}
//   synthesis: x_{2m+e} = sum_u h_{e+2u} a_{(m-u) mod N/2} + g_{e+2u} d_{(m-u) mod N/2}
// In place: every thread first computes its outputs into registers, then the
// block synchronises and writes them back.
// ---------------------------------------------------------------------------
template <typename T, bool ROWS, bool SYNTH>
__device__ void dwt_pass(T *buf, int pitch, int lgN, const Geo<T> &G)
{
    const int N = 1 << lgN, half = N >> 1, total = N * half, Lh = G.n_taps >> 1;
    const int lgh = lgN - 1;
    const int stride = ROWS ? 1 : pitch;
    T o0[kPairs], o1[kPairs];
#pragma unroll
    for (int t = 0; t < kPairs; t++) {
        const int idx = threadIdx.x + t * blockDim.x;
        o0[t] = o1[t] = T(0);
        if (idx < total) {
            // ROWS: line = row, m along the row; COLS: line = column (consecutive
            // threads take consecutive columns), m along the column
            const int line = ROWS ? (idx >> lgh) : (idx & (N - 1));
            const int m = ROWS ? (idx & (half - 1)) : (idx >> lgN);
            const T *base = ROWS ? buf + line * pitch : buf + line;
            T x0 = 0, x1 = 0;
            if (SYNTH) {
#pragma unroll
                for (int u = 0; u < kMaxT / 2; u++) {
                    if (u < Lh) {
                        const int k = (m - u) & (half - 1);
                        const T a = base[k * stride], d = base[(half + k) * stride];
                        x0 += G.h[2 * u] * a + G.g[2 * u] * d;
                        x1 += G.h[2 * u + 1] * a + G.g[2 * u + 1] * d;
                    }
                }
            } else {
#pragma unroll
                for (int u = 0; u < kMaxT; u++) {
                    if (u < 2 * Lh) {
                        const T v = base[((2 * m + u) & (N - 1)) * stride];
                        x0 += G.h[u] * v;
                        x1 += G.g[u] * v;
                    }
                }
            }
            o0[t] = x0;
            o1[t] = x1;
        }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kPairs; t++) {
        const int idx = threadIdx.x + t * blockDim.x;
        if (idx < total) {
            const int line = ROWS ? (idx >> lgh) : (idx & (N - 1));
            const int m = ROWS ? (idx & (half - 1)) : (idx >> lgN);
            T *base = ROWS ? buf + line * pitch : buf + line;
            const int p0 = SYNTH ? 2 * m : m, p1 = SYNTH ? 2 * m + 1 : half + m;
            base[p0 * stride] = o0[t];
            base[p1 * stride] = o1[t];
        }
    }
    __syncthreads();
}

template <typename T>
__device__ void idwt2(T *buf, int lgn, int J, const Geo<T> &G)
{
    for (int t = J - 1; t >= 0; t--) {
        dwt_pass<T, false, true>(buf, 1 << lgn, lgn - t, G);
        dwt_pass<T, true, true>(buf, 1 << lgn, lgn - t, G);
    }
}

template <typename T>
__device__ void fdwt2(T *buf, int lgn, int J, const Geo<T> &G)
{
    for (int t = 0; t < J; t++) {
        dwt_pass<T, true, false>(buf, 1 << lgn, lgn - t, G);
        dwt_pass<T, false, false>(buf, 1 << lgn, lgn - t, G);
    }
}

// ---------------------------------------------------------------------------
// Layer phase 1: coefficients -> nodal values, nodal = W^T coef / delta_l.
// `load(e)` returns the coefficient of global index e (and may fuse vector
// updates); runs for the layers owned by this CTA.
// ---------------------------------------------------------------------------
template <typename T, typename S, class Load>
__device__ void layer_idwt(const Args<T, S> &A, T *buf, Load load)
{
    const Geo<T> &G = A.geo;
    for (int l = blockIdx.x; l < G.L; l += gridDim.x) {
        const int n = G.lay_n[l], nn = n * n;
        const long off = G.lay_off[l];
        for (int e = threadIdx.x; e < nn; e += blockDim.x) buf[e] = load(off + e);
        __syncthreads();
        idwt2<T>(buf, G.lay_lg[l], G.lay_J[l], G);
        const T sc = G.inv_delta[l];
        for (int e = threadIdx.x; e < nn; e += blockDim.x) A.nodal[off + e] = Cv<S>::st(buf[e] * sc);
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
__device__ typename AccT<T>::type wfs_phase(const Args<T, S> &A, T *sm)
{
    typedef typename AccT<T>::type Acc;
    const Geo<T> &G = A.geo;
    const int TS = G.tile, H = TS + 2, SB = TS + 1, m = G.m, ns = G.ns;
    const int per_g = G.tiles_x * G.tiles_x, total = G.G * per_g;
    T *phi = sm;                         // [L][H*H] per-layer contributions (OP)
    T *sx = sm + (size_t)G.L * H * H;    // [SB*SB]
    T *sy = sx + SB * SB;
    Acc ws = 0;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int g = w / per_g, tt = w - g * per_g;
        const int i0 = (tt / G.tiles_x) * TS, j0 = (tt % G.tiles_x) * TS;
        if (!RHS) {
            // per (layer, halo node) bilinear value
            for (int e = threadIdx.x; e < G.L * H * H; e += blockDim.x) {
                const int l = e / (H * H), loc = e - l * H * H;
                const int i = i0 - 1 + loc / H, j = j0 - 1 + loc % H;
                T v = 0;
                if (i >= 0 && i < m && j >= 0 && j < m) {
                    const int bx = ((g * G.L + l) * 2 + 0) * m, by = ((g * G.L + l) * 2 + 1) * m;
                    const int kx = __ldg(G.fk + bx + j), ky = __ldg(G.fk + by + i);
                    const T wx = __ldg(G.fw + bx + j), wy = __ldg(G.fw + by + i);
                    const int n = G.lay_n[l];
                    const S *Lp = A.nodal + G.lay_off[l] + (long)ky * n + kx;
                    const T v00 = Cv<S>::ld(ldcg(Lp)), v01 = Cv<S>::ld(ldcg(Lp + 1));
                    const T v10 = Cv<S>::ld(ldcg(Lp + n)), v11 = Cv<S>::ld(ldcg(Lp + n + 1));
                    v = (T(1) - wy) * ((T(1) - wx) * v00 + wx * v01) + wy * ((T(1) - wx) * v10 + wx * v11);
                }
                phi[e] = v;
            }
            __syncthreads();
            for (int loc = threadIdx.x; loc < H * H; loc += blockDim.x) {
                T s = 0;
                for (int l = 0; l < G.L; l++) s += phi[l * H * H + loc];
                phi[loc] = s;
            }
            __syncthreads();
        }
        // weighted slopes of subapertures (i0-1 .. i0+TS-1) x (j0-1 .. j0+TS-1)
        for (int e = threadIdx.x; e < SB * SB; e += blockDim.x) {
            const int a = e / SB, b = e - a * SB;
            const int i = i0 - 1 + a, j = j0 - 1 + b;
            T vx = 0, vy = 0;
            if (i >= 0 && i < ns && j >= 0 && j < ns) {
                const T wgt = __ldg(G.wmask + (size_t)g * ns * ns + i * ns + j);
                if (RHS) {
                    const S *sg = A.slopes + (size_t)g * 2 * ns * ns;
                    vx = wgt * Cv<S>::ld(sg[i * ns + j]);
                    vy = wgt * Cv<S>::ld(sg[ns * ns + i * ns + j]);
                } else {
                    const T p00 = phi[a * H + b], p01 = phi[a * H + b + 1];
                    const T p10 = phi[(a + 1) * H + b], p11 = phi[(a + 1) * H + b + 1];
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
        for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) {
            const int a = e / TS + 1, b = e % TS + 1;  // subaperture-local (i, j) of node (i0+a-1, j0+b-1)
            const int i = i0 + a - 1, j = j0 + b - 1;
            if (i < m && j < m) {
                const T v = T(0.5) * (sx[a * SB + b - 1] - sx[a * SB + b] + sx[(a - 1) * SB + b - 1] -
                                      sx[(a - 1) * SB + b] + sy[(a - 1) * SB + b] - sy[a * SB + b] +
                                      sy[(a - 1) * SB + b - 1] - sy[a * SB + b - 1]);
                A.psi[(size_t)g * m * m + i * m + j] = Cv<S>::st(v);
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
template <typename T, typename S>
__device__ void band_gather(const Args<T, S> &A, T *sm)
{
    const Geo<T> &G = A.geo;
    const int m = G.m, RC = G.rows_chunk;
    for (int w = blockIdx.x; w < G.nbands; w += gridDim.x) {
        const int l = __ldg(G.band_layer + w), a0 = __ldg(G.band_row0 + w), BR = __ldg(G.band_rows + w);
        const int n = G.lay_n[l], nout = BR * n;
        T *ps = sm;               // [RC][m]   staged psi rows
        T *Tb = sm + RC * m;      // [RC][n]   x-contracted rows
        T acc = 0;
        const int oa = threadIdx.x / n, ob = threadIdx.x - oa * n;  // owned output (a0 + oa, ob)
        for (int g = 0; g < G.G; g++) {
            const int bx = (g * G.L + l) * 2, by = bx + 1;
            const int ilo = __ldg(G.band_ilo + g * G.nbands + w), ihi = __ldg(G.band_ihi + g * G.nbands + w);
            const S *psg = A.psi + (size_t)g * m * m;
            for (int c0 = ilo; c0 < ihi; c0 += RC) {
                const int rows = min(RC, ihi - c0);
                for (int e = threadIdx.x; e < rows * m; e += blockDim.x)
                    ps[e] = Cv<S>::ld(ldcg(psg + (size_t)c0 * m + e));
                __syncthreads();
                for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
                    const int i = e / n, b = e - i * n;
                    const int jlo = __ldg(G.alo + bx * FEWHA_MAX_GRID + b);
                    const int jhi = __ldg(G.ahi + bx * FEWHA_MAX_GRID + b);
                    T v = 0;
                    for (int j = jlo; j < jhi; j++) {
                        const T w0 = __ldg(G.fw + bx * m + j);
                        const T wx = (__ldg(G.fk + bx * m + j) == b) ? T(1) - w0 : w0;
                        v += wx * ps[i * m + j];
                    }
                    Tb[e] = v;
                }
                __syncthreads();
                if (oa < BR) {
                    const int a = a0 + oa;
                    const int rlo = max(__ldg(G.alo + by * FEWHA_MAX_GRID + a), c0);
                    const int rhi = min(__ldg(G.ahi + by * FEWHA_MAX_GRID + a), c0 + rows);
                    for (int i = rlo; i < rhi; i++) {
                        const T w0 = __ldg(G.fw + by * m + i);
                        const T wy = (__ldg(G.fk + by * m + i) == a) ? T(1) - w0 : w0;
                        acc += wy * Tb[(i - c0) * n + ob];
                    }
                }
                __syncthreads();
            }
        }
        if (oa < BR && threadIdx.x < nout) A.u[G.lay_off[l] + (long)(a0 + oa) * n + ob] = acc;
    }
}

// ---------------------------------------------------------------------------
// Layer phase 2: W u / delta_l per layer; `store(e, value)` consumes each
// coefficient (u was written by band_gather in another CTA: L2 loads).
// ---------------------------------------------------------------------------
template <typename T, typename S, class Store>
__device__ void layer_fdwt(const Args<T, S> &A, T *buf, Store store)
{
    const Geo<T> &G = A.geo;
    for (int l = blockIdx.x; l < G.L; l += gridDim.x) {
        const int n = G.lay_n[l], nn = n * n;
        const long off = G.lay_off[l];
        for (int e = threadIdx.x; e < nn; e += blockDim.x) buf[e] = ldcg(A.u + off + e);
        __syncthreads();
        fdwt2<T>(buf, G.lay_lg[l], G.lay_J[l], G);
        const T sc = G.inv_delta[l];
        for (int e = threadIdx.x; e < nn; e += blockDim.x) store(off + e, buf[e] * sc);
        __syncthreads();
    }
}

// Element range of this CTA for vector phases.
__device__ __forceinline__ void cta_range(long n, long &lo, long &hi)
{
    long chunk = (n + gridDim.x - 1) / gridDim.x;
    lo = (long)blockIdx.x * chunk;
    hi = lo + chunk < n ? lo + chunk : n;
}

}  // namespace fewha
