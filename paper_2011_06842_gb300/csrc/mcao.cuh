// MCAO fitting onto several deformable mirrors (Sec. 5: the 9-layer MCAO case
// solves the fitting equation with an unpreconditioned CG of 4 iterations).
// Normal equations N a = b, N = sum_t P^DM_t^T P^DM_t, b = sum_t P^DM_t^T
// P^L_t W^{-1} c over the fitting directions t; P^DM_t and P^L_t are bilinear
// projections of the mirrors and layers onto the pupil nodes (no cone).
//
// One cooperative kernel per fit; phases separated by the bounded grid
// barrier, deterministic two-stage reductions (one partial per CTA):
//   0: y_t = P^L_t nodal - P^DM_t a0           (pupil maps, all directions)
//   1: r = sum_t P^DM_t^T y_t, p = r, (r, r)    (gather over each actuator's
//                                                 pupil-node ranges, no atomics;
//                                                 one lane per direction)
//   per iteration: y = P^DM p | q = N p, (p, q) | a += alpha p, r -= alpha q,
//   (r, r) | p = r + beta p
#pragma once

#include "device.cuh"

namespace fewha {

template <typename T, typename S>
struct McaoArgs {
    const S *nodal;                         // W^{-1} c, layer after layer
    int L, D, ndir, m, nmax;
    long lay_off[FEWHA_MAX_LAYERS];
    int lay_n[FEWHA_MAX_LAYERS];
    int dm_n[FEWHA_MAX_DM];
    long dm_off[FEWHA_MAX_DM + 1];
    const int *lk;                          // [t][l][axis][m] lower layer node of pupil node j
    const T *lw;                            //                 its fractional position
    const int *dk;                          // [t][d][axis][m] lower actuator of pupil node j
    const T *dw;
    const int *alo, *ahi;                   // [t][d][axis][nmax] pupil nodes an actuator reaches
    T *a, *r, *p, *q, *y;                   // y: [t][m][m]
    double *part;                           // [2][kMaxCtas] partial sums
    Record *rec;
    int iters;
    unsigned long long timeout_ns;
};

// bilinear sample of an n x n grid; L2 loads (the mirror vectors change
// between phases of the same launch)
template <typename T, typename V>
__device__ __forceinline__ T mcao_bilinear(const V *g, int n, int kx, int ky, T wx, T wy)
{
    const V *p = g + (long)ky * n + kx;
    const T v00 = Cv<V>::ld(ldcg(p)), v01 = Cv<V>::ld(ldcg(p + 1));
    const T v10 = Cv<V>::ld(ldcg(p + n)), v11 = Cv<V>::ld(ldcg(p + n + 1));
    return (T(1) - wy) * ((T(1) - wx) * v00 + wx * v01) + wy * ((T(1) - wx) * v10 + wx * v11);
}

// y_t(node) = [sum_l layer_l] - sum_d mirror_d (v), every direction t
template <typename T, typename S>
__device__ __forceinline__ void mcao_project(const McaoArgs<T, S> &M, const T *v, bool with_layers)
{
    const int m = M.m, mm = m * m;
    const long total = (long)M.ndir * mm;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int t = (int)(e / mm), rem = (int)(e - (long)t * mm), iy = rem / m, ix = rem - iy * m;
        T lay = 0;
        if (with_layers) {
#pragma unroll 3
            for (int l = 0; l < M.L; l++) {
                const int bx = ((t * M.L + l) * 2) * m, by = bx + m;
                lay += mcao_bilinear<T, S>(M.nodal + M.lay_off[l], M.lay_n[l], __ldg(M.lk + bx + ix),
                                           __ldg(M.lk + by + iy), __ldg(M.lw + bx + ix), __ldg(M.lw + by + iy));
            }
        }
        T dm = 0;
#pragma unroll 3
        for (int d = 0; d < M.D; d++) {
            const int bx = ((t * M.D + d) * 2) * m, by = bx + m;
            dm += mcao_bilinear<T, T>(v + M.dm_off[d], M.dm_n[d], __ldg(M.dk + bx + ix), __ldg(M.dk + by + iy),
                                      __ldg(M.dw + bx + ix), __ldg(M.dw + by + iy));
        }
        M.y[e] = with_layers ? lay - dm : dm;
    }
}

// (P^DM_t^T y_t) at actuator e for the directions t = t0, t0 + kDirLanes, ...,
// gathered over the pupil nodes its hat functions reach (rows v, columns u)
constexpr int kDirLanes = 8;  // lanes that share one actuator, one direction each

template <typename T, typename S>
__device__ __forceinline__ T mcao_adjoint_at(const McaoArgs<T, S> &M, long e, int t0)
{
    int d = 0;
    while (e >= M.dm_off[d + 1]) d++;
    const int n = M.dm_n[d], loc = (int)(e - M.dm_off[d]), iy = loc / n, ix = loc - iy * n;
    const int m = M.m;
    T s = 0;
    for (int t = t0; t < M.ndir; t += kDirLanes) {
        const int bx = ((t * M.D + d) * 2) * m, by = bx + m;
        const int rx = ((t * M.D + d) * 2) * M.nmax, ry = rx + M.nmax;
        const int u0 = __ldg(M.alo + rx + ix), u1 = __ldg(M.ahi + rx + ix);
        const int v0 = __ldg(M.alo + ry + iy), v1 = __ldg(M.ahi + ry + iy);
        const T *yt = M.y + (long)t * m * m;
        for (int v = v0; v < v1; v++) {
            const T fy = __ldg(M.dw + by + v);
            const T wy = __ldg(M.dk + by + v) == iy ? T(1) - fy : fy;
            T row = 0;
            for (int u = u0; u < u1; u++) {
                const T fx = __ldg(M.dw + bx + u);
                const T wx = __ldg(M.dk + bx + u) == ix ? T(1) - fx : fx;
                row += wx * ldcg(yt + (long)v * m + u);
            }
            s += wy * row;
        }
    }
    return s;
}

// For every actuator (kDirLanes lanes each, 32 / kDirLanes actuators per warp):
// v = sum_t P^DM_t^T y_t, the lanes' direction sums added in a fixed shuffle
// tree; body(e, v) runs on the group's first lane.
template <typename T, typename S, class Body>
__device__ __forceinline__ void mcao_adjoint(const McaoArgs<T, S> &M, long nact, Body body)
{
    const int lane = threadIdx.x & 31, sub = lane & (kDirLanes - 1);
    const long warp = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
    const long nwarps = ((long)gridDim.x * blockDim.x) >> 5, per = 32 / kDirLanes;
    for (long eb = warp * per; eb < nact; eb += nwarps * per) {  // uniform over the warp
        const long e = eb + lane / kDirLanes;
        T v = e < nact ? mcao_adjoint_at<T, S>(M, e, sub) : T(0);
#pragma unroll
        for (int o = kDirLanes / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (sub == 0 && e < nact) body(e, v);
    }
}

// The adjoint phases and the vector updates map actuators to threads
// differently, so every read of a, r, p, q goes through L2.
template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_mcao_fit(const __grid_constant__ McaoArgs<T, S> M)
{
    typedef typename AccT<T>::type Acc;
    __shared__ double sred[kSred];
    __shared__ double red[2];
    const int nc = gridDim.x, rank = blockIdx.x;
    const long nact = M.dm_off[M.D];
    const long g0 = blockIdx.x * (long)blockDim.x + threadIdx.x, gs = (long)gridDim.x * blockDim.x;
    const int slot_rr[1] = {0}, slot_pq[1] = {1};
    auto sync = [&]() { return grid_sync(M.rec, M.timeout_ns, nc, rank); };
    auto reduce1 = [&](int slot) {
        reduce_ranges(M.part, nc, {slot, 1, red});
        return red[0];
    };

    mcao_project<T, S>(M, M.a, true);  // y = phi - P^DM a0
    if (!sync()) return;
    {
        Acc acc[1] = {0};
        mcao_adjoint<T, S>(M, nact, [&](long e, T r) {
            M.r[e] = r;
            M.p[e] = r;
            acc[0] += (Acc)r * (Acc)r;
        });
        block_partials<1>(acc, M.part, slot_rr, sred, rank);
    }
    if (!sync()) return;
    double rr = reduce1(0);
    for (int it = 0; it < M.iters; it++) {
        if (rr == 0.0) break;  // uniform: every CTA reduced the same partials
        mcao_project<T, S>(M, M.p, false);  // y = P^DM p
        if (!sync()) return;
        {
            Acc acc[1] = {0};
            mcao_adjoint<T, S>(M, nact, [&](long e, T q) {
                M.q[e] = q;
                acc[0] += (Acc)ldcg(M.p + e) * (Acc)q;
            });
            block_partials<1>(acc, M.part, slot_pq, sred, rank);
        }
        if (!sync()) return;
        const double pq = reduce1(1);
        const T alpha = (T)(rr / pq);
        {
            Acc acc[1] = {0};
            for (long e = g0; e < nact; e += gs) {
                M.a[e] = ldcg(M.a + e) + alpha * ldcg(M.p + e);
                const T r = ldcg(M.r + e) - alpha * ldcg(M.q + e);
                M.r[e] = r;
                acc[0] += (Acc)r * (Acc)r;
            }
            block_partials<1>(acc, M.part, slot_rr, sred, rank);
        }
        if (!sync()) return;
        const double rr_new = reduce1(0);
        const T beta = (T)(rr_new / rr);
        for (long e = g0; e < nact; e += gs) M.p[e] = ldcg(M.r + e) + beta * ldcg(M.p + e);
        rr = rr_new;
        if (!sync()) return;
    }
}

}  // namespace fewha
