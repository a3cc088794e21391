// Solver phases of one reconstructor time step (Ramlau & Stadler,
// Algorithm 3 right-hand side and residual steps, then Algorithm 1 / 2).
//
// Scalar work is arranged for this GPU's FP64 units (dependent FP64
// latency ~64 cycles, a division ~430): every phase reduces the partial
// sums it needs in one round (one warp per slot); the iteration scalars
// avoid divisions on the critical path (1/rz_k and 1/(p_m, q_m) are stored
// when they become known); the k x k Cholesky factor of the recycled basis'
// Gram matrix is computed once per time step by one warp of the last CTA
// while the right-hand side is being assembled.
#pragma once
#include "device.cuh"

namespace fewha {

// Recycled basis of the previous solve (bank ob) and the bank this solve fills.
struct Basis {
    int ob, nb, kv, head;
};

template <typename T, typename S>
__device__ __forceinline__ Basis basis_info(const Args<T, S> &A)
{
    Basis b;
    b.ob = ldcgi(A.meta) & 1;
    b.nb = 1 - b.ob;
    int cnt = ldcgi(A.meta + 1);
    b.kv = A.augmented ? (cnt < A.kcap ? cnt : A.kcap) : 0;
    b.head = ldcgi(A.meta + 2);
    return b;
}

// slot of old basis vector j (0 = oldest .. kv-1 = newest)
template <typename T, typename S>
__device__ __forceinline__ int old_slot(const Args<T, S> &A, const Basis &b, int j)
{
    int s = (b.head - b.kv + 1 + j) % A.kcap;
    return s < 0 ? s + A.kcap : s;
}

template <typename T, typename S>
__device__ __forceinline__ const T *oldP(const Args<T, S> &A, const Basis &b, int j)
{
    return A.P + ((size_t)b.ob * A.kcap + old_slot(A, b, j)) * A.geo.n;
}
template <typename T, typename S>
__device__ __forceinline__ const T *oldQ(const Args<T, S> &A, const Basis &b, int j)
{
    return A.Q + ((size_t)b.ob * A.kcap + old_slot(A, b, j)) * A.geo.n;
}
template <typename T, typename S>
__device__ __forceinline__ T *newP(const Args<T, S> &A, const Basis &b, int k)
{
    return A.P + ((size_t)b.nb * A.kcap + (k % A.kcap)) * A.geo.n;
}
template <typename T, typename S>
__device__ __forceinline__ T *newQ(const Args<T, S> &A, const Basis &b, int k)
{
    return A.Q + ((size_t)b.nb * A.kcap + (k % A.kcap)) * A.geo.n;
}

// Shared scalars of a phase (every CTA derives them from the same partials).
struct Scal {
    double red[2 * kK + 16];       // reduced partials
    double gram[kK * kK];          // reduced Gram matrix
    double L[kK * kK], dinv[kK];   // Cholesky factor (copy of the record's)
    double tau[kK];                // projection coefficients
    double rz, beta, mu, rr, bb, pq, alpha, rinv_pqm, rinv;
    int stop;
};

// Loads the Cholesky factor of the old basis (computed during R2) into shared memory.
template <typename T, typename S>
__device__ void load_factor(const Args<T, S> &A, int kv, Scal &sc)
{
    for (int e = threadIdx.x; e < kv * kv; e += blockDim.x) sc.L[e] = ldcgd(A.rec->L + e);
    if (threadIdx.x < kv) sc.dinv[threadIdx.x] = ldcgd(A.rec->dinv + threadIdx.x);
    if (threadIdx.x == 0) sc.rinv_pqm = ldcgd(&A.rec->rinv_pqm);
    __syncthreads();
}

// ---------------------------------------------------------------------------
// R1 (second part): Gram matrix G_ij = (p_i, q_j) of the old basis.  The
// CTA's slice of the kv directions p and q is staged in shared memory (one
// latency round), then one warp per entry sums it.
// ---------------------------------------------------------------------------
template <typename T, typename S>
__device__ __noinline__ void phase_gram(const Args<T, S> &A, const Basis &b, T *sm, int sm_elems)
{
    typedef typename AccT<T>::type Acc;
    constexpr int W = VW<T>::W;
    long lo, hi;
    cta_range_vec(A.geo.n, W, A.vrank(), A.ncta, lo, hi);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int kv = b.kv, nslot = kv * kv, nvec = 2 * kv;
    const int CH = (sm_elems / nvec) / W * W;  // elements of the slice staged at once
    Acc acc[(kK * kK + 31) / 32];
    for (int i = 0; i < (kK * kK + 31) / 32; i++) acc[i] = 0;
    for (long c0 = lo; c0 < hi; c0 += CH) {
        const int len = (int)min((long)CH, hi - c0);
        for (int v = threadIdx.x; v < nvec * (len / W); v += blockDim.x) {
            const int vec = v / (len / W), o = (v - vec * (len / W)) * W;
            const T *src = vec < kv ? oldP(A, b, vec) : oldQ(A, b, vec - kv);
            T x[W];
            vld_nc(src + c0 + o, x);
            vst(sm + vec * CH + o, x);
        }
        __syncthreads();
        for (int s2 = warp, t = 0; s2 < nslot; s2 += nw, t++) {
            const T *X = sm + (s2 / kv) * CH, *Y = sm + (kv + s2 % kv) * CH;
            Acc a = 0;
            for (int e = lane; e < len; e += 32) a += (Acc)X[e] * (Acc)Y[e];
            acc[t] += a;
        }
        __syncthreads();
    }
    for (int s2 = warp, t = 0; s2 < nslot; s2 += nw, t++) {
        const Acc a = warp_sum_t(acc[t]);
        if (lane == 0) A.part[(size_t)(kSlotGram + s2) * kMaxCtas + A.vrank()] = (double)a;
    }
    __syncthreads();
}

// R2 side task of the last CTA: Cholesky factor of G (symmetrised) and
// 1/(p_m, q_m), into the record.
template <typename T, typename S>
__device__ __noinline__ void phase_factor(const Args<T, S> &A, const Basis &b, Scal &sc)
{
    const int kv = b.kv;
    reduce_ranges(A.part, A.ncta, {kSlotGram, kv * kv, sc.gram});
    if (threadIdx.x < 32) {
        const bool ok = warp_cholesky(kv, sc.gram, sc.L, sc.dinv);
        if (threadIdx.x == 0) {
            if (!ok) set_status(A.rec, FEWHA_ERR_NOT_SPD);
            A.rec->rinv_pqm = 1.0 / ldcgd(A.pq + b.ob * A.kcap + b.head);
        }
        for (int e = threadIdx.x; e < kv * kv; e += 32) A.rec->L[e] = sc.L[e];
        if (threadIdx.x < kv) A.rec->dinv[threadIdx.x] = sc.dinv[threadIdx.x];
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// R3: right-hand side b = W^{-T} u / delta (u = P^T Gamma^T C s from the
// preceding phases) and the warm-restart residual of Algorithm 3,
// r0 = (b - b_prev) + r_prev;  b_prev <- b.
// ---------------------------------------------------------------------------
template <typename T, typename S>
__device__ __noinline__ void phase_rhs_fdwt(const Args<T, S> &A, T *sm, double *sred)
{
    typedef typename AccT<T>::type Acc;
    constexpr int W = VW<T>::W;
    Acc acc[2] = {0, 0};
    layer_fdwt<T, S>(A, sm, [&](long e, const T (&b)[W]) {
        T bp[W], rp[W], r0[W];
        vld(A.b_prev + e, bp);
        vld_cg(A.r + e, rp);
#pragma unroll
        for (int i = 0; i < W; i++) {
            r0[i] = (b[i] - bp[i]) + rp[i];
            acc[0] += (Acc)b[i] * (Acc)b[i];
            acc[1] += (Acc)r0[i] * (Acc)r0[i];
        }
        vst(A.b_prev + e, b);
        vst(A.r + e, r0);
    });
    const int slots[2] = {kSlotR2, kSlotR2 + 1};
    block_partials<2>(acc, A.part, slots, sred, A.vrank());
}

// INIT1: P^T r0 (Algorithm 2 initial projection), per CTA slice.
template <typename T, typename S>
__device__ __noinline__ void phase_ptr(const Args<T, S> &A, const Basis &b, double *sred)
{
    typedef typename AccT<T>::type Acc;
    constexpr int W = VW<T>::W;
    long lo, hi;
    cta_range_vec(A.geo.n, W, A.vrank(), A.ncta, lo, hi);
    Acc acc[kK];
    for (int j = 0; j < kK; j++) acc[j] = 0;
    for (long e = lo + (long)threadIdx.x * W; e < hi; e += (long)blockDim.x * W) {
        T rv[W];
        vld_cg(A.r + e, rv);
        for (int j = 0; j < b.kv; j++) {
            T pj[W];
            vld_nc(oldP(A, b, j) + e, pj);
#pragma unroll
            for (int i = 0; i < W; i++) acc[j] += (Acc)pj[i] * (Acc)rv[i];
        }
    }
    int slots[kK];
    for (int j = 0; j < kK; j++) slots[j] = kSlotGram + kK * kK + j;
    block_partials<kK>(acc, A.part, slots, sred, A.vrank());
}

// INIT2: c += P sigma, r -= Q sigma with sigma = G^{-1} P^T r0; then the
// partial sums (q_j, z), (r, z), (r, r) with z = J^{-1} r.
template <typename T, typename S>
__device__ __noinline__ void phase_init(const Args<T, S> &A, const Basis &b, Scal &sc, double *sred)
{
    const int kv = b.kv;
    reduce_ranges(A.part, A.ncta, {kSlotGram + kK * kK, kv, sc.red});
    load_factor(A, kv, sc);
    if (threadIdx.x < 32) warp_chol_solve(kv, sc.L, sc.dinv, sc.red, sc.tau);
    __syncthreads();
    typedef typename AccT<T>::type Acc;
    constexpr int W = VW<T>::W;
    long lo, hi;
    cta_range_vec(A.geo.n, W, A.vrank(), A.ncta, lo, hi);
    Acc acc[kK + 2];
    for (int j = 0; j < kK + 2; j++) acc[j] = 0;
    for (long e = lo + (long)threadIdx.x * W; e < hi; e += (long)blockDim.x * W) {
        T cv[W], rv[W], jv[W];
        vld(A.c + e, cv);
        vld_cg(A.r + e, rv);
        vld_nc(A.geo.invJ + e, jv);
        for (int j = 0; j < kv; j++) {
            const T sj = (T)sc.tau[j];
            T pj[W], qj[W];
            vld_nc(oldP(A, b, j) + e, pj);
            vld_nc(oldQ(A, b, j) + e, qj);
#pragma unroll
            for (int i = 0; i < W; i++) {
                cv[i] += sj * pj[i];
                rv[i] -= sj * qj[i];
            }
        }
        vst(A.c + e, cv);
        vst(A.r + e, rv);
        T z[W];
#pragma unroll
        for (int i = 0; i < W; i++) {
            z[i] = jv[i] * rv[i];
            acc[kK] += (Acc)rv[i] * (Acc)z[i];
            acc[kK + 1] += (Acc)rv[i] * (Acc)rv[i];
        }
        for (int j = 0; j < kv; j++) {
            T qj[W];
            vld_nc(oldQ(A, b, j) + e, qj);
#pragma unroll
            for (int i = 0; i < W; i++) acc[j] += (Acc)qj[i] * (Acc)z[i];
        }
    }
    int slots[kK + 2];
    for (int j = 0; j < kK; j++) slots[j] = kSlotInit + j;
    slots[kK] = kSlotInit + kK;
    slots[kK + 1] = kSlotInit + kK + 1;
    block_partials<kK + 2>(acc, A.part, slots, sred, A.vrank());
}

// ---------------------------------------------------------------------------
// U_k: iteration scalars, then the direction update, element-parallel over all
// CTAs (each CTA its own element range):
//   k = 0: p_0 = z_0 - P G^{-1} Q^T z_0 (Algorithm 2) or z_0 (Algorithm 1)
//   k > 0: p_k = (z_k - mu p_m) + beta p_{k-1},  mu = (z_k, q_m)/(p_m, q_m),
//          rz_k = (r_k, z_k) - mu (r_k, p_m),  beta = rz_k / rz_{k-1}
//          (all-directions variant: z_k - P G^{-1} Q^T z_k)
// Returns false (uniformly) when the stopping test holds before iteration k.
// CTA 0 records rz_k (k > 0) and ||b||^2 (k = 0).  Partial sums of
// (alpha D p_k, p_k) and (r_k, p_k) go to the A slots.
// ---------------------------------------------------------------------------
template <typename T, typename S>
__device__ __noinline__ bool phase_U(const Args<T, S> &A, const Basis &b, int k, Scal &sc, double *sred,
                                     bool scalars_in_sc = false)
{
    const int kv = b.kv;
    double *red = sc.red;
    if (k == 0) {
        // red: [0] bb, [1] rr (R3), [2..2+kv) Q^T z, [2+kv] rz, [3+kv] rr (INIT2)
        if (kv > 0)
            reduce_ranges(A.part, A.ncta, {kSlotR2, 2, red}, {kSlotInit, kv, red + 2},
                          {kSlotInit + kK, 2, red + 2 + kv});
        else
            reduce_ranges(A.part, A.ncta, {kSlotR2, 2, red});
        if (kv > 0) {
            load_factor(A, kv, sc);
            if (threadIdx.x < 32) warp_chol_solve(kv, sc.L, sc.dinv, red + 2, sc.tau);
        }
        if (threadIdx.x == 0) {
            sc.bb = red[0];
            sc.rr = kv > 0 ? red[3 + kv] : red[1];
            sc.beta = 0.0;
            sc.mu = 0.0;
            if (A.vrank() == 0) A.rec->bb = sc.bb;
        }
    } else {
        // red: [0] rz, [1] zq, [2] rp, [3] rr (E_{k-1}); [4..4+kv) Q^T z, [4+kK..) P^T r
        const int e0 = kSlotE + ((k - 1) & 1) * kSlotEStride;
        if (A.recycle_all && kv > 0)
            reduce_ranges(A.part, A.ncta, {e0, 4, red}, {e0 + 4, kv, red + 4}, {e0 + 4 + kK, kv, red + 4 + kK});
        else
            reduce_ranges(A.part, A.ncta, {e0, 4, red});
        if (kv > 0 && A.recycle_all) {
            load_factor(A, kv, sc);
            if (threadIdx.x < 32) warp_chol_solve(kv, sc.L, sc.dinv, red + 4, sc.tau);
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            double rz = red[0];
            sc.mu = 0.0;
            if (kv > 0) {
                if (A.recycle_all) {
                    for (int j = 0; j < kv; j++) rz -= sc.tau[j] * red[4 + kK + j];
                } else {
                    sc.mu = red[1] * (scalars_in_sc ? sc.rinv_pqm : ldcgd(&A.rec->rinv_pqm));
                    rz -= sc.mu * red[2];
                }
            }
            sc.rz = rz;
            sc.rr = red[3];
            // 1/rz_{k-1}, ||b||^2, 1/(p_m, q_m): kept in shared memory by the
            // persistent kernel, else read from the record
            if (!scalars_in_sc) sc.bb = ldcgd(&A.rec->bb);
            sc.beta = rz * (scalars_in_sc ? sc.rinv : ldcgd(A.rec->rinv + (k - 1)));
            if (A.vrank() == 0) A.rec->rz[k] = rz;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sc.stop = (A.rtol > 0.0 && sc.rr <= A.rtol * A.rtol * sc.bb) ? 1 : 0;
        if (sc.stop && A.vrank() == 0) {
            A.rec->iters = k;
            A.rec->done = 1;
        }
    }
    __syncthreads();
    if (sc.stop) return false;

    const T beta = (T)sc.beta, mu = (T)sc.mu;
    T *pk = newP(A, b, k);
    const T *pprev = k > 0 ? newP(A, b, k - 1) : nullptr;
    const T *pm = kv > 0 ? oldP(A, b, kv - 1) : nullptr;
    const bool proj_all = (k == 0) || A.recycle_all;
    typedef typename AccT<T>::type Acc;
    constexpr int W = VW<T>::W;
    Acc acc[2] = {0, 0};
    long lo, hi;
    cta_range_vec(A.geo.n, W, A.vrank(), A.ncta, lo, hi);
    for (long e = lo + (long)threadIdx.x * W; e < hi; e += (long)blockDim.x * W) {
        T p[W];
        T rv[W], jv[W], ad[W], pp[W];
        vld_cg(A.r + e, rv);
        vld_nc(A.geo.invJ + e, jv);
        vld_nc(A.geo.alpha_d + e, ad);
        if (k > 0) vld(pprev + e, pp);
#pragma unroll
        for (int i = 0; i < W; i++) p[i] = jv[i] * rv[i];
        if (kv > 0) {
            if (proj_all) {
                for (int j = 0; j < kv; j++) {
                    T pj[W];
                    const T tj = (T)sc.tau[j];
                    vld_nc(oldP(A, b, j) + e, pj);
#pragma unroll
                    for (int i = 0; i < W; i++) p[i] -= tj * pj[i];
                }
            } else {
                T pmv[W];
                vld_nc(pm + e, pmv);
#pragma unroll
                for (int i = 0; i < W; i++) p[i] -= mu * pmv[i];
            }
        }
#pragma unroll
        for (int i = 0; i < W; i++) {
            if (k > 0) p[i] += beta * pp[i];
            acc[0] += (Acc)ad[i] * (Acc)p[i] * (Acc)p[i];
            acc[1] += (Acc)rv[i] * (Acc)p[i];
        }
        vst(pk + e, p);  // p_k into its basis slot
    }
    const int slots[2] = {kSlotA + (k & 1) * 2, kSlotA + (k & 1) * 2 + 1};
    block_partials<2>(acc, A.part, slots, sred, A.vrank());
    return true;
}

// ---------------------------------------------------------------------------
// A_k: nodal layers = W^{-1} p_k, one CTA per layer (p_k from U_k, written by
// other CTAs: L2 loads).
// ---------------------------------------------------------------------------
template <typename T, typename S>
__device__ __noinline__ void phase_A(const Args<T, S> &A, const Basis &b, int k, T *sm)
{
    constexpr int W = VW<T>::W;
    const T *pk = newP(A, b, k);
    layer_idwt<T, S>(A, sm, [&](long e, T (&p)[W]) { vld_cg(pk + e, p); });
}

// ---------------------------------------------------------------------------
// C_k: scalars of iteration k and u = P^T psi.  (p_k, q_k) comes from the
// forward pass: sum w s^2 (WFS phase) + sum alpha d p^2 (U phase), equal to
// (p_k, M p_k) by Eq. M.  alpha_k = rz_k / (p_k, q_k) and 1/rz_k are
// computed by two threads at once.  Returns false (uniformly) on rz == 0
// (converged) or breakdown; CTA 0 records alpha_k, 1/rz_k and (p_k, q_k).
// ---------------------------------------------------------------------------
template <typename T, typename S>
__device__ __noinline__ bool phase_C(const Args<T, S> &A, const Basis &b, int k, T *sm, Scal &sc,
                                     bool rz_in_sc = false)
{
    double *red = sc.red;  // [0] ws, [1] pd, [2] rz0 (k = 0)
    reduce_ranges(A.part, A.ncta, {kSlotB + (k & 1), 1, red}, {kSlotA + (k & 1) * 2, k == 0 ? 2 : 1, red + 1});
    if (threadIdx.x == 0) {
        // rz_k: from U_k in this CTA's shared memory (persistent kernel) or the record
        sc.rz = k == 0 ? red[2] : (rz_in_sc ? sc.rz : ldcgd(A.rec->rz + k));
        sc.pq = red[0] + red[1];
    }
    __syncthreads();
    if (threadIdx.x == 0) sc.alpha = sc.rz / sc.pq;
    if (threadIdx.x == 32) sc.rinv = red[3] = 1.0 / sc.rz;
    __syncthreads();
    if (threadIdx.x == 0) {
        sc.stop = 0;
        if (sc.rz == 0.0) {
            sc.stop = 1;
        } else if (!(sc.pq > 0.0) || !isfinite(sc.pq) || !isfinite(sc.rz)) {
            sc.stop = 1;
            if (A.vrank() == 0) set_status(A.rec, FEWHA_ERR_BREAKDOWN);
        }
        if (A.vrank() == 0) {
            if (sc.stop) {
                A.rec->iters = k;
                A.rec->done = 1;
            } else {
                A.rec->rz[k] = sc.rz;
                A.rec->rinv[k] = red[3];
                A.rec->alpha[k] = sc.alpha;
                A.pq[b.nb * A.kcap + (k % A.kcap)] = sc.pq;
            }
        }
    }
    __syncthreads();
    if (sc.stop) return false;
    band_gather<T, S>(A, sm);
    return true;
}

// D_k: wq = W^{-T} u / delta (E_k adds alpha D p_k to form q_k).
template <typename T, typename S>
__device__ __noinline__ void phase_D(const Args<T, S> &A, T *sm)
{
    constexpr int W = VW<T>::W;
    layer_fdwt<T, S>(A, sm, [&](long e, const T (&v)[W]) { vst(A.wq + e, v); });
}

// E_k: q_k = wq + alpha D p_k (stored in the basis slot), c += alpha p,
// r -= alpha q, and the inner products of the next step.
template <typename T, typename S, bool ALL>
__device__ __noinline__ void phase_E_impl(const Args<T, S> &A, const Basis &b, int k, double *sred,
                                         const double *alpha_sc)
{
    const T alpha = (T)(alpha_sc ? *alpha_sc : ldcgd(A.rec->alpha + k));
    const T *pk = newP(A, b, k);
    T *qk = newQ(A, b, k);
    const int kv = b.kv;
    const T *pm = kv > 0 ? oldP(A, b, kv - 1) : nullptr;
    const T *qm = kv > 0 ? oldQ(A, b, kv - 1) : nullptr;
    constexpr int W = VW<T>::W;
    long lo, hi;
    cta_range_vec(A.geo.n, W, A.vrank(), A.ncta, lo, hi);
    typedef typename AccT<T>::type Acc;
    const bool last = kv > 0 && !ALL;
    const bool all = kv > 0 && ALL;
    constexpr int NA = ALL ? 4 + 2 * kK : 4;
    Acc acc[NA];
    for (int i = 0; i < NA; i++) acc[i] = 0;
    for (long e = lo + (long)threadIdx.x * W; e < hi; e += (long)blockDim.x * W) {
        T p[W], wq[W], ad[W], c[W], r[W], jv[W], q[W], z[W];
        vld_cg(pk + e, p);
        vld_cg(A.wq + e, wq);
        vld_nc(A.geo.alpha_d + e, ad);
        vld(A.c + e, c);
        vld_cg(A.r + e, r);
        vld_nc(A.geo.invJ + e, jv);
        T pmv[W], qmv[W];
        if (last) {
            vld_nc(pm + e, pmv);
            vld_nc(qm + e, qmv);
        }
#pragma unroll
        for (int i = 0; i < W; i++) {
            q[i] = wq[i] + ad[i] * p[i];
            c[i] += alpha * p[i];
            r[i] -= alpha * q[i];
            z[i] = jv[i] * r[i];
            acc[0] += (Acc)r[i] * (Acc)z[i];
            if (last) {
                acc[1] += (Acc)z[i] * (Acc)qmv[i];
                acc[2] += (Acc)r[i] * (Acc)pmv[i];
            }
            acc[3] += (Acc)r[i] * (Acc)r[i];
        }
        vst(qk + e, q);
        vst(A.c + e, c);
        vst(A.r + e, r);
        if constexpr (ALL) {
            if (all) {
                for (int j = 0; j < kv; j++) {
                    T qj[W], pj[W];
                    vld_nc(oldQ(A, b, j) + e, qj);
                    vld_nc(oldP(A, b, j) + e, pj);
#pragma unroll
                    for (int i = 0; i < W; i++) {
                        acc[4 + j] += (Acc)z[i] * (Acc)qj[i];
                        acc[4 + kK + j] += (Acc)r[i] * (Acc)pj[i];
                    }
                }
            }
        }
    }
    const int e0 = kSlotE + (k & 1) * kSlotEStride;
    int slots[NA];
    for (int i = 0; i < NA; i++) slots[i] = e0 + i;
    block_partials<NA>(acc, A.part, slots, sred, A.vrank());
}

template <typename T, typename S>
__device__ void phase_E(const Args<T, S> &A, const Basis &b, int k, double *sred, const double *alpha_sc = nullptr)
{
    if (A.recycle_all)
        phase_E_impl<T, S, true>(A, b, k, sred, alpha_sc);
    else
        phase_E_impl<T, S, false>(A, b, k, sred, alpha_sc);
}

// Stats and the recycled-basis metadata for the next time step (CTA 0).
template <typename T, typename S>
__device__ __noinline__ void phase_finish(const Args<T, S> &A, const Basis &b, int K, Scal &sc)
{
    double *red = sc.red;  // [0] bb, [1] rr (R3), [2] rz, [3] rr (last E or INIT2)
    if (K > 0)
        reduce_ranges(A.part, A.ncta, {kSlotR2, 2, red}, {kSlotE + ((K - 1) & 1) * kSlotEStride, 1, red + 2},
                      {kSlotE + ((K - 1) & 1) * kSlotEStride + 3, 1, red + 3});
    else if (b.kv > 0)
        reduce_ranges(A.part, A.ncta, {kSlotR2, 2, red}, {kSlotInit + kK, 2, red + 2});
    else
        reduce_ranges(A.part, A.ncta, {kSlotR2, 2, red});
    if (threadIdx.x == 0) {
        const double bb = red[0];
        const double rr = (K > 0 || b.kv > 0) ? red[3] : red[1];
        const double rz = (K > 0 || b.kv > 0) ? red[2] : 0.0;
        fewha_stats st;
        st.status = ldcgi(&A.rec->status);
        st.iterations = K;
        st.bnorm = sqrt(bb);
        st.rel_res = bb > 0 ? sqrt(rr / bb) : 0.0;
        st.rz = rz;
        int count = ldcgi(A.meta + 1);
        if (K > 0 && st.status == FEWHA_OK) {
            A.meta[0] = b.nb;
            count = K < A.kcap ? K : A.kcap;
            A.meta[1] = count;
            A.meta[2] = (K - 1) % A.kcap;
        }
        A.meta[3] = ldcgi(A.meta + 3) + 1;
        st.basis_count = count;
        st.pad = 0;
        if (A.stats) *A.stats = st;
    }
}

}  // namespace fewha
