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

// Addresses of the old basis directions p_j, q_j (j < kv) in shared memory, so
// that loops over j can have all their loads in flight at once (one DRAM round
// trip instead of kv: the basis is cold after the previous frame).
template <typename T, typename S>
__device__ __forceinline__ void basis_table(const Args<T, S> &A, const Basis &b, const T **sp, const T **sq)
{
    if (threadIdx.x < b.kv) {
        sp[threadIdx.x] = oldP(A, b, threadIdx.x);
        sq[threadIdx.x] = oldQ(A, b, threadIdx.x);
    }
    __syncthreads();
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
__device__ __forceinline__ void phase_gram(const Args<T, S> &A, const Basis &b, T *sm, int sm_elems)
{
    typedef typename AccT<T>::type Acc;
    constexpr int W = VW<T>::W;
    long lo, hi;
    cta_range_vec(A.geo.n, W, A.vrank(), A.ncta, lo, hi);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int kv = b.kv, nslot = kv * kv, nvec = 2 * kv;
    const int CH = (sm_elems / nvec) / W * W;  // elements of the slice staged at once
    __shared__ const T *sp[kK], *sq[kK];
    basis_table(A, b, sp, sq);
    // warp w sums slots w, w + nw, w + 2 nw, ...: at most kGramT of them
    // (nw = kThreads / 32 warps; k = FEWHA_MAX_K gives kK^2 slots)
    constexpr int kGramT = (kK * kK + kThreads / 32 - 1) / (kThreads / 32);
    Acc acc[kGramT];
    for (int i = 0; i < kGramT; i++) acc[i] = 0;
    for (long c0 = lo; c0 < hi; c0 += CH) {
        const int len = (int)min((long)CH, hi - c0);
        const int nv = len / W, total = nvec * nv;
        constexpr int U = 4;  // vectors in flight per thread
        for (int v0 = threadIdx.x; v0 < total; v0 += U * blockDim.x) {
            T x[U][W];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int v = v0 + u * blockDim.x;
                if (v < total) {
                    const int vec = v / nv, o = (v - vec * nv) * W;
                    vld_nc((vec < kv ? sp[vec] : sq[vec - kv]) + c0 + o, x[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int v = v0 + u * blockDim.x;
                if (v < total) {
                    const int vec = v / nv, o = (v - vec * nv) * W;
                    vst(sm + vec * CH + o, x[u]);
                }
            }
        }
        __syncthreads();
        for (int s2 = warp, t = 0; s2 < nslot && t < kGramT; s2 += nw, t++) {
            const T *X = sm + (s2 / kv) * CH, *Y = sm + (kv + s2 % kv) * CH;
            Acc a = 0;
            for (int e = lane; e < len; e += 32) a += (Acc)X[e] * (Acc)Y[e];
            acc[t] += a;
        }
        __syncthreads();
    }
    for (int s2 = warp, t = 0; s2 < nslot && t < kGramT; s2 += nw, t++) {
        const Acc a = warp_sum_t(acc[t]);
        if (lane == 0) A.part[(size_t)(kSlotGram + s2) * kMaxCtas + A.vrank()] = (double)a;
    }
    __syncthreads();
}

// R2 side task of the last CTA: Cholesky factor of G (symmetrised) and
// 1/(p_m, q_m), into the record.
template <typename T, typename S>
__device__ __forceinline__ void phase_factor(const Args<T, S> &A, const Basis &b, Scal &sc)
{
    const int kv = b.kv;
    reduce_wide(A.part, A.ncta, kSlotGram, kv * kv, sc.gram);
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

// INIT2: c += P sigma, r -= Q sigma with sigma = G^{-1} P^T r0; then the
// partial sums (q_j, z), (r, z), (r, r) with z = J^{-1} r.
template <typename T, typename S>
__device__ __forceinline__ void phase_init(const Args<T, S> &A, const Basis &b, Scal &sc, double *sred)
{
    const int kv = b.kv;
    __shared__ const T *sp[kK], *sq[kK];
    basis_table(A, b, sp, sq);
    // the Cholesky factor (written during R2) is loaded while P^T r0 is reduced
    const int nf = kv * kv;
    double fv = 0.0;
    if (threadIdx.x < nf)
        fv = ldcgd(A.rec->L + threadIdx.x);
    else if (threadIdx.x < nf + kv)
        fv = ldcgd(A.rec->dinv + threadIdx.x - nf);
    reduce_ranges(A.part, A.ncta, {kSlotGram + kK * kK, kv, sc.red});
    if (threadIdx.x < nf)
        sc.L[threadIdx.x] = fv;
    else if (threadIdx.x < nf + kv)
        sc.dinv[threadIdx.x - nf] = fv;
    __syncthreads();
    if (threadIdx.x < 32) warp_chol_solve(kv, sc.L, sc.dinv, sc.red, sc.tau);
    __syncthreads();
    typedef typename AccT<T>::type Acc;
    constexpr int W = VW<T>::W;
    long lo, hi;
    cta_range_vec(A.geo.n, W, A.vrank(), A.ncta, lo, hi);
    Acc acc[kK + 2];
#pragma unroll
    for (int j = 0; j < kK + 2; j++) acc[j] = 0;
    constexpr int CJ = 8;  // directions loaded at once
    for (long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
        T cv = A.c[e], rv = ldcg(A.r + e);
        const T jv = __ldg(A.geo.invJ + e);
        for (int j0 = 0; j0 < kv; j0 += CJ) {
            T pj[CJ], qj[CJ];
#pragma unroll
            for (int t = 0; t < CJ; t++) {
                const bool in = j0 + t < kv;
                pj[t] = in ? __ldg(sp[j0 + t] + e) : T(0);
                qj[t] = in ? __ldg(sq[j0 + t] + e) : T(0);
            }
#pragma unroll
            for (int t = 0; t < CJ; t++) {
                if (j0 + t < kv) {
                    const T sj = (T)sc.tau[j0 + t];
                    cv += sj * pj[t];
                    rv -= sj * qj[t];
                }
            }
        }
        A.c[e] = cv;
        A.r[e] = rv;
        const T z = jv * rv;
        acc[kK] += (Acc)rv * (Acc)z;
        acc[kK + 1] += (Acc)rv * (Acc)rv;
        // q_j again (now from L1)
        T qj[kK];
#pragma unroll
        for (int j = 0; j < kK; j++) qj[j] = j < kv ? __ldg(sq[j] + e) : T(0);
#pragma unroll
        for (int j = 0; j < kK; j++) acc[j] += (Acc)qj[j] * (Acc)z;
    }
    int slots[kK + 2];
    for (int j = 0; j < kK; j++) slots[j] = kSlotInit + j;
    slots[kK] = kSlotInit + kK;
    slots[kK + 1] = kSlotInit + kK + 1;
    block_partials<kK + 2>(acc, A.part, slots, sred, A.vrank());
}

// ---------------------------------------------------------------------------
// Element loops of the fused phases.  Every layer's top-left (n/2)^2 block (the
// approximation part of the finest wavelet level) belongs to the layer's CTA,
// which transforms it in shared memory; every other coefficient to the CTA
// whose element range holds it.
// ---------------------------------------------------------------------------
template <typename T, typename F>
__device__ __forceinline__ void for_detail_vectors(const Geo<T> &G, long lo, long hi, F body)
{
    constexpr int W = VW<T>::W;
    int l = 0;
    for (long e = lo + (long)threadIdx.x * W; e < hi; e += (long)blockDim.x * W) {
        while (e >= G.lay_off[l + 1]) l++;
        const long loc = e - G.lay_off[l];
        const int h = G.lay_n[l] >> 1;
        if ((int)(loc >> G.lay_lg[l]) < h && (int)(loc & (G.lay_n[l] - 1)) < h) continue;
        body(e);
    }
}

// Two ways to run the layers' transforms, chosen per instance:
//   split (at least twice as many CTAs as layers): the finest level is tiled
//     over all CTAs (A2, D1); the first L CTAs own one layer's (n/2)^2 block
//     each, run its coarser levels in shared memory and take no detail
//     coefficients (the block transforms are then the critical path);
//   whole (fewer CTAs, e.g. the small instances of a batch): each layer's CTA
//     updates the whole layer, runs every level in shared memory and updates
//     the layer again after the forward transform; A2 and D1 are empty, so an
//     iteration has four grid barriers instead of six.
template <typename T, typename S>
__device__ __forceinline__ bool split_levels(const Args<T, S> &A)
{
    return A.ncta >= 2 * A.geo.L;
}

// body(global element, index in the (n/2)^2 block), one W-vector per call
template <typename T, typename F>
__device__ __forceinline__ void for_block_vectors(const Geo<T> &G, int l, F body)
{
    constexpr int W = VW<T>::W;
    const int n = G.lay_n[l], h = n >> 1, lgh = G.lay_lg[l] - 1, nv = h * h / W;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
        const int be = v * W;
        body(G.lay_off[l] + (long)(be >> lgh) * n + (be & (h - 1)), be);
    }
}

// ---------------------------------------------------------------------------
// UA1_k: iteration scalars, the direction update (element-parallel), and the
// coarser synthesis levels of W^{-1} p_k on each layer's (n/2)^2 block (the
// layer's CTA updates that block straight into shared memory):
//   k = 0: p_0 = z_0 - P G^{-1} Q^T z_0 (Algorithm 2) or z_0 (Algorithm 1)
//   k > 0: p_k = (z_k - mu p_m) + beta p_{k-1},  mu = (z_k, q_m)/(p_m, q_m),
//          rz_k = (r_k, z_k) - mu (r_k, p_m),  beta = rz_k / rz_{k-1}
//          (all-directions variant: z_k - P G^{-1} Q^T z_k)
// Returns false (uniformly) when the stopping test holds before iteration k.
// CTA 0 records rz_k (k > 0) and ||b||^2 (k = 0).  Partial sums of
// (alpha D p_k, p_k) and (r_k, p_k) go to the A slots; the blocks' level-1
// approximations go to A.ll for A2_k.
// ---------------------------------------------------------------------------
template <typename T, typename S>
__device__ __forceinline__ bool phase_UA1(const Args<T, S> &A, const Basis &b, int k, T *buf, Scal &sc,
                                       double *sred, bool scalars_in_sc = false,
                                       typename AccT<T>::type *defer = nullptr)
{
    typedef typename AccT<T>::type Acc;
    constexpr int W = VW<T>::W;
    const int kv = b.kv;
    const Geo<T> &G = A.geo;
    const bool split = split_levels(A);
    const bool proj_all = (k == 0) || A.recycle_all;
    // The first vector this thread updates (split form, k > 0, last-direction
    // projection) has its operands loaded before the reduction below, which
    // hides their latency.
    long pe = -1;
    T pr[W], pj[W], pa[W], ppp[W], ppm[W];
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
        if (split && !A.recycle_all) {
            if (A.vrank() < G.L) {
                const int l = A.vrank(), h = G.lay_n[l] >> 1, lgh = G.lay_lg[l] - 1, be = threadIdx.x * W;
                if (be < h * h) pe = G.lay_off[l] + (long)(be >> lgh) * G.lay_n[l] + (be & (h - 1));
            } else {
                long lo, hi;
                cta_range_vec(G.n, W, A.vrank() - G.L, A.ncta - G.L, lo, hi);
                if (lo + (long)threadIdx.x * W < hi) pe = lo + (long)threadIdx.x * W;
            }
            if (pe >= 0) {
                vld_cg(A.r + pe, pr);
                vld_nc(G.invJ + pe, pj);
                vld_nc(G.alpha_d + pe, pa);
                vld_cg(newP(A, b, k - 1) + pe, ppp);
                if (kv > 0) vld_nc(oldP(A, b, kv - 1) + pe, ppm);
            }
        }
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
    if (threadIdx.x == 0) {  // the thread that set rr and bb
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
    __shared__ const T *sp[kK], *sq[kK];
    if (proj_all && kv > 0) basis_table(A, b, sp, sq);
    Acc acc[2] = {0, 0};
    const T *pprev = k > 0 ? newP(A, b, k - 1) : nullptr;
    const T *pm = kv > 0 ? oldP(A, b, kv - 1) : nullptr;
    // PF: the call may take the prefetched operands (split form only, so that
    // the whole-layer loop does not keep them live across its transforms)
    auto update_t = [&](bool use_pf, long e, T (&p)[W]) {
        T rv[W], jv[W], ad[W], pp[W], pmv[W];
        if (use_pf && e == pe) {
#pragma unroll
            for (int i = 0; i < W; i++) {
                rv[i] = pr[i];
                jv[i] = pj[i];
                ad[i] = pa[i];
                pp[i] = ppp[i];
                pmv[i] = ppm[i];
            }
        } else {
            vld_cg(A.r + e, rv);
            vld_nc(G.invJ + e, jv);
            vld_nc(G.alpha_d + e, ad);
            if (k > 0) vld_cg(pprev + e, pp);
            if (kv > 0 && !proj_all) vld_nc(pm + e, pmv);
        }
#pragma unroll
        for (int i = 0; i < W; i++) p[i] = jv[i] * rv[i];
        if (kv > 0) {
            if (proj_all) {
                for (int j = 0; j < kv; j++) {
                    T pj[W];
                    const T tj = (T)sc.tau[j];
                    vld_nc(sp[j] + e, pj);
#pragma unroll
                    for (int i = 0; i < W; i++) p[i] -= tj * pj[i];
                }
            } else {
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
    };
    auto update = [&](long e, T (&p)[W]) { update_t(true, e, p); };
    auto update_np = [&](long e, T (&p)[W]) { update_t(false, e, p); };
    if (split) {
        // one layer per layer CTA (ncta >= 2L); the others take the details
        if (A.vrank() < G.L) {
            const int l = A.vrank(), h = G.lay_n[l] >> 1, lgh = G.lay_lg[l] - 1;
            for_block_vectors(G, l, [&](long e, int be) {
                T p[W];
                update(e, p);
                const int s0 = spad(be, lgh);
#pragma unroll
                for (int i = 0; i < W; i++) buf[s0 + i] = p[i];
            });
            __syncthreads();
            idwt2<T>(buf, G.pingpong ? buf + h * (h + 1) : buf, lgh, G.lay_J[l] - 1, G);
            T *ll = A.ll + G.ll_off[l];
            for (int v = threadIdx.x; v < h * h / W; v += blockDim.x) {
                const int be = v * W, s0 = spad(be, lgh);
                T x[W];
#pragma unroll
                for (int i = 0; i < W; i++) x[i] = buf[s0 + i];
                vst(ll + be, x);
            }
            __syncthreads();
        } else {
            long lo, hi;
            cta_range_vec(G.n, W, A.vrank() - G.L, A.ncta - G.L, lo, hi);
            for_detail_vectors(G, lo, hi, [&](long e) {
                T p[W];
                update(e, p);
            });
        }
    } else {
        for (int l = A.vrank(); l < G.L; l += A.ncta) {
            // whole layer: p_k into shared memory, all levels, nodal = W^{-1} p_k
            const int n = G.lay_n[l], lgn = G.lay_lg[l], nv = n * n / W;
            const long off = G.lay_off[l];
            for (int v = threadIdx.x; v < nv; v += blockDim.x) {
                T p[W];
                update_np(off + (long)v * W, p);
                const int s0 = spad(v * W, lgn);
#pragma unroll
                for (int i = 0; i < W; i++) buf[s0 + i] = p[i];
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
    if (defer) {
        // the caller adds them to a later phase's block reduction
        defer[0] = acc[0];
        defer[1] = acc[1];
    } else {
        const int slots[2] = {kSlotA + (k & 1) * 2, kSlotA + (k & 1) * 2 + 1};
        block_partials<2>(acc, A.part, slots, sred, A.vrank());
    }
    return true;
}

// ---------------------------------------------------------------------------
// C_k: scalars of iteration k and u = P^T psi.  (p_k, q_k) comes from the
// forward pass: sum w s^2 (WFS phase) + sum alpha d p^2 (U phase), equal to
// (p_k, M p_k) by Eq. M.  alpha_k = rz_k / (p_k, q_k) and 1/rz_k are
// computed by two threads at once.  Returns false (uniformly) on rz == 0
// (converged) or breakdown; CTA 0 records alpha_k, 1/rz_k and (p_k, q_k).
// ---------------------------------------------------------------------------
template <typename T, typename S>
__device__ __forceinline__ bool phase_C(const Args<T, S> &A, const Basis &b, int k, T *sm, Scal &sc,
                                     bool rz_in_sc = false)
{
    double *red = sc.red;  // [0] ws, [1] pd, [2] rz0 (k = 0)
    const BandHdr hdr = band_header(A, A.vrank());  // in flight during the reduction
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
    band_gather<T, S>(A, sm, &hdr);
    return true;
}

// ---------------------------------------------------------------------------
// Split layer transforms.  The finest level of the periodic 2-D DWT is a local
// stencil: a level-1 coefficient pair depends on an L x L window of the layer
// (analysis), and a pair of nodal values on Lh x Lh windows of the four level-1
// subbands (synthesis).  That level runs in tiles of kFineTile x kFineTile
// coefficient pairs on all CTAs; only the coarser levels, on the (n/2)^2
// approximation block, stay on one CTA per layer.  Same sums in the same order
// as the single-CTA transform (rows then columns for analysis, columns then
// rows for synthesis).
// ---------------------------------------------------------------------------
constexpr int kFineTile = 16;

// Work item w -> layer l and tile origin (in coefficient pairs); false past the end.
template <typename T>
__device__ __forceinline__ bool fine_tile(const Geo<T> &G, int w, int &l, int &p0y, int &p0x)
{
    for (l = 0; l < G.L; l++) {
        const int h = G.lay_n[l] >> 1, nt = (h + kFineTile - 1) / kFineTile;
        if (w < nt * nt) {
            p0y = (w / nt) * kFineTile;
            p0x = (w % nt) * kFineTile;
            return true;
        }
        w -= nt * nt;
    }
    return false;
}

// D1: level-1 analysis of u; the three detail bands are final coefficients of
// W^{-T} u / delta (into wq), the approximation block goes to A.ll.
template <typename T, typename S, int L>
__device__ void fine_analysis(const Args<T, S> &A, T *sm)
{
    const Geo<T> &G = A.geo;
    const Taps<T, L> tp = load_taps<T, L>(G);
    int l, p0y, p0x;
    for (int w = A.vrank(); fine_tile(G, w, l, p0y, p0x); w += A.ncta) {
        const int n = G.lay_n[l], h = n >> 1;
        const int ty = min(kFineTile, h - p0y), tx = min(kFineTile, h - p0x);
        const int IR = 2 * ty + L - 2, IC = 2 * tx + L - 2, MC = 2 * tx;
        T *in = sm, *mid = sm + IR * IC;
        const T *u = A.u + G.lay_off[l];
        for (int e = threadIdx.x; e < IR * IC; e += blockDim.x) {
            const int r = e / IC, c = e - r * IC;
            in[e] = ldcg(u + (long)((2 * p0y + r) & (n - 1)) * n + ((2 * p0x + c) & (n - 1)));
        }
        __syncthreads();
        for (int e = threadIdx.x; e < IR * tx; e += blockDim.x) {  // rows
            const int r = e / tx, k = e - r * tx;
            const T *x = in + r * IC + 2 * k;
            T a = 0, d = 0;
#pragma unroll
            for (int t = 0; t < L; t++) {
                a += tp.h[t] * x[t];
                d += tp.g[t] * x[t];
            }
            mid[r * MC + k] = a;
            mid[r * MC + tx + k] = d;
        }
        __syncthreads();
        const T sc = G.inv_delta[l];
        T *wq = A.wq + G.lay_off[l];
        T *ll = A.ll + G.ll_off[l];
        for (int e = threadIdx.x; e < ty * MC; e += blockDim.x) {  // columns
            const int k = e / MC, c = e - k * MC;
            const T *x = mid + 2 * k * MC + c;
            T a = 0, d = 0;
#pragma unroll
            for (int t = 0; t < L; t++) {
                a += tp.h[t] * x[t * MC];
                d += tp.g[t] * x[t * MC];
            }
            const int row = p0y + k;
            if (c < tx) {  // low x: LL (unscaled, coarser levels follow) and HL
                ll[(long)row * h + p0x + c] = a;
                wq[(long)(h + row) * n + p0x + c] = d * sc;
            } else {       // high x: LH and HH
                const int q = h + p0x + (c - tx);
                wq[(long)row * n + q] = a * sc;
                wq[(long)(h + row) * n + q] = d * sc;
            }
        }
        __syncthreads();
    }
}

// A2: level-1 synthesis of p_k's layers from the approximation block in A.ll
// (A1) and p_k's three detail bands; nodal = W^{-1} p_k.
template <typename T, typename S, int L>
__device__ void fine_synthesis(const Args<T, S> &A, const T *pk, T *sm)
{
    constexpr int Lh = L / 2;
    const Geo<T> &G = A.geo;
    const Taps<T, L> tp = load_taps<T, L>(G);
    int l, p0y, p0x;
    for (int w = A.vrank(); fine_tile(G, w, l, p0y, p0x); w += A.ncta) {
        const int n = G.lay_n[l], h = n >> 1;
        const int ty = min(kFineTile, h - p0y), tx = min(kFineTile, h - p0x);
        const int WR = ty + Lh - 1, WC = tx + Lh - 1, Q = WR * WC;
        T *win = sm;              // [4][WR][WC]: LL, LH, HL, HH windows
        T *mid = sm + 4 * Q;      // [2 ty][2 WC]: columns synthesised, low-x then high-x
        const T *ll = A.ll + G.ll_off[l];
        const T *pl = pk + G.lay_off[l];
        for (int e = threadIdx.x; e < 4 * Q; e += blockDim.x) {
            const int qd = e / Q, r = (e - qd * Q) / WC, c = e - qd * Q - r * WC;
            const int m = (p0y - Lh + 1 + r) & (h - 1), j = (p0x - Lh + 1 + c) & (h - 1);
            T v;
            if (qd == 0)
                v = ldcg(ll + (long)m * h + j);
            else if (qd == 1)
                v = ldcg(pl + (long)m * n + h + j);
            else if (qd == 2)
                v = ldcg(pl + (long)(h + m) * n + j);
            else
                v = ldcg(pl + (long)(h + m) * n + h + j);
            win[e] = v;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 2 * ty * 2 * WC; e += blockDim.x) {  // columns
            const int yy = e / (2 * WC), cc = e - yy * (2 * WC);
            const int i = yy >> 1, ey = yy & 1, half = cc >= WC ? 1 : 0, c = cc - half * WC;
            const T *lo = win + (half ? 1 : 0) * Q + c;  // low y: LL or LH
            const T *hi = win + (half ? 3 : 2) * Q + c;  // high y: HL or HH
            T x = 0;
#pragma unroll
            for (int u = 0; u < Lh; u++) {
                const int r = i + Lh - 1 - u;
                x += tp.h[ey + 2 * u] * lo[r * WC] + tp.g[ey + 2 * u] * hi[r * WC];
            }
            mid[e] = x;
        }
        __syncthreads();
        const T sc = G.inv_delta[l];
        S *nodal = A.nodal + G.lay_off[l];
        for (int e = threadIdx.x; e < 2 * ty * 2 * tx; e += blockDim.x) {  // rows
            const int yy = e / (2 * tx), xx = e - yy * (2 * tx), j = xx >> 1, ex = xx & 1;
            const T *row = mid + yy * 2 * WC;
            T x = 0;
#pragma unroll
            for (int u = 0; u < Lh; u++) {
                const int c = j + Lh - 1 - u;
                x += tp.h[ex + 2 * u] * row[c] + tp.g[ex + 2 * u] * row[WC + c];
            }
            nodal[(long)(2 * p0y + yy) * n + 2 * p0x + xx] = Cv<S>::st(x * sc);
        }
        __syncthreads();
    }
}

// The finest synthesis level of vector x, tiled over all CTAs (split form).
template <typename T, typename S>
__device__ __forceinline__ void phase_fine_synth(const Args<T, S> &A, const T *x, T *sm)
{
    if (!split_levels(A)) return;
    switch (A.geo.n_taps) {
    case 2: fine_synthesis<T, S, 2>(A, x, sm); break;
    case 4: fine_synthesis<T, S, 4>(A, x, sm); break;
    case 6: fine_synthesis<T, S, 6>(A, x, sm); break;
    default: fine_synthesis<T, S, 8>(A, x, sm); break;
    }
}

// A2_k: the finest synthesis level, tiled over all CTAs: nodal = W^{-1} p_k.
template <typename T, typename S>
__device__ __forceinline__ void phase_A2(const Args<T, S> &A, const Basis &b, int k, T *sm)
{
    phase_fine_synth(A, newP(A, b, k), sm);
}

// D1_k: the finest analysis level of u, tiled over all CTAs.
template <typename T, typename S>
__device__ __forceinline__ void phase_D1(const Args<T, S> &A, T *sm)
{
    if (!split_levels(A)) return;
    switch (A.geo.n_taps) {
    case 2: fine_analysis<T, S, 2>(A, sm); break;
    case 4: fine_analysis<T, S, 4>(A, sm); break;
    case 6: fine_analysis<T, S, 6>(A, sm); break;
    default: fine_analysis<T, S, 8>(A, sm); break;
    }
}


// ---------------------------------------------------------------------------
// The last part of W^{-T} u / delta and an element update over it.  Split form
// (after D1): each layer CTA runs the coarser analysis levels of its layer's
// approximation block (from A.ll) in shared memory and calls upd(e, wq) for
// the block's W-vectors with wq taken from there; every other CTA calls it
// for the detail coefficients in its element range with wq from A.wq (D1's
// output).  Whole form: each layer's CTA transforms the whole of u's layer in
// shared memory and calls upd for every W-vector of the layer.
// ---------------------------------------------------------------------------
template <typename T, typename S, class Upd>
__device__ __forceinline__ void analysis_update(const Args<T, S> &A, T *buf, Upd update_w)
{
    constexpr int W = VW<T>::W;
    auto update = [&](long e) {
        T wq[W];
        vld_cg(A.wq + e, wq);
        update_w(e, wq);
    };
    const Geo<T> &G = A.geo;
    if (!split_levels(A)) {
        // whole layer: W^{-T} u / delta in shared memory, then the update of the
        // layer with wq read from there
        for (int l = A.vrank(); l < G.L; l += A.ncta) {
            const int n = G.lay_n[l], lgn = G.lay_lg[l], nv = n * n / W;
            const long off = G.lay_off[l];
#pragma unroll 2
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
            for (int v = threadIdx.x; v < nv; v += blockDim.x) {
                T wq[W];
                const int s0 = spad(v * W, lgn);
#pragma unroll
                for (int i = 0; i < W; i++) wq[i] = buf[s0 + i] * sc;
                update_w(off + (long)v * W, wq);
            }
            __syncthreads();
        }
    }
    // split: the layer's CTA runs the coarser analysis levels of the
    // approximation block (from D1_k), then the update on that block with
    // W^{-T} u / delta taken from shared memory; the other CTAs update the
    // detail coefficients (their wq from D1_k)
    if (split_levels(A)) {
        if (A.vrank() < G.L) {
            const int l = A.vrank(), n = G.lay_n[l], h = n >> 1, lgh = G.lay_lg[l] - 1, nv = h * h / W;
            const T *ll = A.ll + G.ll_off[l];
#pragma unroll 4
            for (int v = threadIdx.x; v < nv; v += blockDim.x) {
                T x[W];
                vld_cg(ll + (long)v * W, x);
                const int s0 = spad(v * W, lgh);
#pragma unroll
                for (int i = 0; i < W; i++) buf[s0 + i] = x[i];
            }
            __syncthreads();
            fdwt2<T>(buf, G.pingpong ? buf + h * (h + 1) : buf, lgh, G.lay_J[l] - 1, G);
            const T sc = G.inv_delta[l];
            for_block_vectors(G, l, [&](long e, int be) {
                T wq[W];
                const int s0 = spad(be, lgh);
#pragma unroll
                for (int i = 0; i < W; i++) wq[i] = buf[s0 + i] * sc;
                update_w(e, wq);
            });
            __syncthreads();
        } else {
            long lo, hi;
            cta_range_vec(G.n, W, A.vrank() - G.L, A.ncta - G.L, lo, hi);
            for_detail_vectors(G, lo, hi, update);
        }
    }
}

// D2E_k: the coarser analysis levels of each layer's approximation block (the
// layer's CTA; W^{-T} u / delta is then complete), and the update
// q_k = wq + alpha D p_k (stored in the basis slot), c += alpha p,
// r -= alpha q with the inner products of the next step (element-parallel;
// each layer's block by its CTA right after its transform).
//
// TR = true (residual replacement after iteration k, same layer transforms):
// with u = P^T Gamma^T C Gamma P W^{-1} c from the preceding phases, the true
// residual r = b - (W^{-T} u / delta + alpha D c) replaces r (b is in b_prev
// since R3), and the same partial sums of the next step are taken from it.
template <typename T, typename S, bool ALL, bool TR = false>
__device__ __forceinline__ void phase_D2E_impl(const Args<T, S> &A, const Basis &b, int k, T *buf, double *sred,
                                           const double *alpha_sc)
{
    const T alpha = TR ? T(0) : (T)(alpha_sc ? *alpha_sc : ldcgd(A.rec->alpha + k));
    const T *pk = TR ? nullptr : newP(A, b, k);
    T *qk = TR ? nullptr : newQ(A, b, k);
    const int kv = b.kv;
    const T *pm = kv > 0 ? oldP(A, b, kv - 1) : nullptr;
    const T *qm = kv > 0 ? oldQ(A, b, kv - 1) : nullptr;
    constexpr int W = VW<T>::W;
    typedef typename AccT<T>::type Acc;
    const bool last = kv > 0 && !ALL;
    const bool all = kv > 0 && ALL;
    constexpr int NA = ALL ? 4 + 2 * kK : 4;
    Acc acc[NA];
    for (int i = 0; i < NA; i++) acc[i] = 0;
    auto update_w = [&](long e, const T (&wq)[W]) {
        T p[W], ad[W], c[W], r[W], jv[W], q[W], z[W];
        T pmv[W], qmv[W];
        if constexpr (TR) {
            vld_cg(A.b_prev + e, r);  // b of this time step
        } else {
            vld_cg(pk + e, p);
            vld_cg(A.r + e, r);
        }
        vld_nc(A.geo.alpha_d + e, ad);
        vld_cg(A.c + e, c);
        vld_nc(A.geo.invJ + e, jv);
        if (last) {
            vld_nc(pm + e, pmv);
            vld_nc(qm + e, qmv);
        }
#pragma unroll
        for (int i = 0; i < W; i++) {
            if constexpr (TR) {
                r[i] -= wq[i] + ad[i] * c[i];  // b - M c
            } else {
                q[i] = wq[i] + ad[i] * p[i];
                c[i] += alpha * p[i];
                r[i] -= alpha * q[i];
            }
            z[i] = jv[i] * r[i];
            acc[0] += (Acc)r[i] * (Acc)z[i];
            if (last) {
                acc[1] += (Acc)z[i] * (Acc)qmv[i];
                acc[2] += (Acc)r[i] * (Acc)pmv[i];
            }
            acc[3] += (Acc)r[i] * (Acc)r[i];
        }
        if constexpr (!TR) {
            vst(qk + e, q);
            vst(A.c + e, c);
        }
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
    };
    analysis_update(A, buf, update_w);
    const int e0 = kSlotE + (k & 1) * kSlotEStride;
    int slots[NA];
    for (int i = 0; i < NA; i++) slots[i] = e0 + i;
    block_partials<NA>(acc, A.part, slots, sred, A.vrank());
}

template <typename T, typename S>
__device__ void phase_D2E(const Args<T, S> &A, const Basis &b, int k, T *buf, double *sred,
                          const double *alpha_sc = nullptr)
{
    if (A.recycle_all)
        phase_D2E_impl<T, S, true>(A, b, k, buf, sred, alpha_sc);
    else
        phase_D2E_impl<T, S, false>(A, b, k, buf, sred, alpha_sc);
}

// ---------------------------------------------------------------------------
// R3 (after D1 of u in the split form; on u in the whole form): the
// right-hand side b = W^{-T} u / delta and the warm-restart residual of
// Algorithm 3, r0 = (b - b_prev) + r_prev, b_prev <- b, with the partial
// sums of ||b||^2 and ||r0||^2 and, when a recycled basis is present, of
// P^T r0 (the first step of Algorithm 2's initial projection) in the same
// pass over the elements.
// ---------------------------------------------------------------------------
// The W-vectors whose update analysis_update gives to this CTA, in the same
// order: its layer's block (split form, layer CTAs), its detail range (split
// form, other CTAs), or its whole layers (whole form).
template <typename T, typename S, class F>
__device__ __forceinline__ void for_updated_vectors(const Args<T, S> &A, F body)
{
    constexpr int W = VW<T>::W;
    const Geo<T> &G = A.geo;
    if (!split_levels(A)) {
        for (int l = A.vrank(); l < G.L; l += A.ncta)
            for (int v = threadIdx.x; v < G.lay_n[l] * G.lay_n[l] / W; v += blockDim.x) body(G.lay_off[l] + (long)v * W);
    } else if (A.vrank() < G.L) {
        for_block_vectors(G, A.vrank(), [&](long e, int) { body(e); });
    } else {
        long lo, hi;
        cta_range_vec(G.n, W, A.vrank() - G.L, A.ncta - G.L, lo, hi);
        for_detail_vectors(G, lo, hi, body);
    }
}

// P^T r0 partial sums of R3 for up to KV recycled directions, together with
// the ||b||^2 and ||r0||^2 partials already in acc.
template <typename T, typename S, int KV>
__device__ __noinline__ void rhs_ptr_pass(const Args<T, S> &A, const Basis &b,
                                             const typename AccT<T>::type (&acc)[2], double *sred)
{
    typedef typename AccT<T>::type Acc;
    constexpr int W = VW<T>::W;
    const int kv = b.kv;
    __shared__ const T *sp[kK], *sq[kK];
    basis_table(A, b, sp, sq);
    Acc pr[2 + KV];
    pr[0] = acc[0];
    pr[1] = acc[1];
#pragma unroll
    for (int j = 0; j < KV; j++) pr[2 + j] = 0;
    for_updated_vectors(A, [&](long e) {
        T r0[W];
        vld_cg(A.r + e, r0);
        constexpr int CJ = 2;  // directions loaded at once
#pragma unroll
        for (int j0 = 0; j0 < KV; j0 += CJ) {
            if (j0 < kv) {
                T pj[CJ][W];
#pragma unroll
                for (int t = 0; t < CJ; t++)
                    if (j0 + t < kv) vld_nc(sp[j0 + t] + e, pj[t]);
#pragma unroll
                for (int t = 0; t < CJ; t++)
                    if (j0 + t < kv) {
#pragma unroll
                        for (int i = 0; i < W; i++) pr[2 + j0 + t] += (Acc)pj[t][i] * (Acc)r0[i];
                    }
            }
        }
    });
    int slots[2 + KV];
    slots[0] = kSlotR2;
    slots[1] = kSlotR2 + 1;
#pragma unroll
    for (int j = 0; j < KV; j++) slots[2 + j] = kSlotGram + kK * kK + j;
    block_partials<2 + KV>(pr, A.part, slots, sred, A.vrank());
}

template <typename T, typename S, bool RIS>
__device__ __forceinline__ void phase_rhs_update(const Args<T, S> &A, const Basis &b, T *buf, double *sred)
{
    typedef typename AccT<T>::type Acc;
    constexpr int W = VW<T>::W;
    const int kv = b.kv;
    Acc acc[2] = {0, 0};
    if constexpr (RIS) {
        // the state already holds b (in b_prev) and r0: partial sums only
        for_updated_vectors(A, [&](long e) {
            T bv[W], r0[W];
            vld_cg(A.b_prev + e, bv);
            vld_cg(A.r + e, r0);
#pragma unroll
            for (int i = 0; i < W; i++) {
                acc[0] += (Acc)bv[i] * (Acc)bv[i];
                acc[1] += (Acc)r0[i] * (Acc)r0[i];
            }
        });
    } else analysis_update(A, buf, [&](long e, const T (&bv)[W]) {
        T bp[W], rp[W], r0[W];
        vld(A.b_prev + e, bp);
        vld_cg(A.r + e, rp);
#pragma unroll
        for (int i = 0; i < W; i++) {
            r0[i] = (bv[i] - bp[i]) + rp[i];
            acc[0] += (Acc)bv[i] * (Acc)bv[i];
            acc[1] += (Acc)r0[i] * (Acc)r0[i];
        }
        vst(A.b_prev + e, bv);
        vst(A.r + e, r0);
    });
    if (kv == 0) {
        const int slots[2] = {kSlotR2, kSlotR2 + 1};
        block_partials<2>(acc, A.part, slots, sred, A.vrank());
        return;
    }
    // P^T r0 over the same elements (each thread rereads the r0 it wrote),
    // in a second pass so that its accumulators are not live across the
    // layer transforms; accumulators sized for the basis in use
    if (kv <= 8)
        rhs_ptr_pass<T, S, 8>(A, b, acc, sred);
    else
        rhs_ptr_pass<T, S, kK>(A, b, acc, sred);
}

// ---------------------------------------------------------------------------
// Residual replacement after iteration k (every true_res_every-th iteration;
// not in the paper, whose Algorithms 1-3 keep the recurrence residual):
// r <- b - M c with one operator application of c, run on the working-
// precision view of the arguments (TrView below), phases
//   TU   nodal = W^{-1} c: coarser levels of c's (n/2)^2 block on the layer
//        CTAs into A.ll (split form), or every level per layer (whole form)
//   TA2  the finest synthesis level tiled over all CTAs (split form)
//   TB   WFS phase (P_g, Gamma, C_eta^{-1}, Gamma^T)
//   TC   P^T gather
//   TD1  the finest analysis level of u (split form)
//   TE   the coarser analysis levels, then r = b - (W^{-T} u / delta + alpha D c),
//        z = J^{-1} r and the partial sums of the next step (replacing D2E_k's)
// Iteration k+1 then takes its scalars from the true residual.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void phase_TU(const Args<T, T> &A, T *buf)
{
    constexpr int W = VW<T>::W;
    const Geo<T> &G = A.geo;
    if (split_levels(A)) {
        if (A.vrank() < G.L) {
            const int l = A.vrank(), h = G.lay_n[l] >> 1, lgh = G.lay_lg[l] - 1;
            for_block_vectors(G, l, [&](long e, int be) {
                T x[W];
                vld_cg(A.c + e, x);
                const int s0 = spad(be, lgh);
#pragma unroll
                for (int i = 0; i < W; i++) buf[s0 + i] = x[i];
            });
            __syncthreads();
            idwt2<T>(buf, G.pingpong ? buf + h * (h + 1) : buf, lgh, G.lay_J[l] - 1, G);
            T *ll = A.ll + G.ll_off[l];
            for (int v = threadIdx.x; v < h * h / W; v += blockDim.x) {
                const int be = v * W, s0 = spad(be, lgh);
                T x[W];
#pragma unroll
                for (int i = 0; i < W; i++) x[i] = buf[s0 + i];
                vst(ll + be, x);
            }
            __syncthreads();
        }
    } else {
        layer_idwt<T, T>(A, buf, [&](long e, T (&x)[W]) { vld_cg(A.c + e, x); });
    }
}

template <typename T>
__device__ void phase_TE(const Args<T, T> &A, const Basis &b, int k, T *buf, double *sred)
{
    if (A.recycle_all)
        phase_D2E_impl<T, T, true, true>(A, b, k, buf, sred, nullptr);
    else
        phase_D2E_impl<T, T, false, true>(A, b, k, buf, sred, nullptr);
}

// The residual replacement's view of the arguments: the same arguments with
// the operator's nodal layers and adjoint wavefronts in the working precision
// T.  With S == T that is the arguments themselves; otherwise a copy in
// shared memory whose nodal / psi point at the T-typed buffers.
template <typename T, typename S>
struct TrView {
    __device__ static const Args<T, T> *get(const Args<T, S> &A)
    {
        static_assert(sizeof(Args<T, T>) == sizeof(Args<T, S>), "same layout");
        __shared__ __align__(16) Args<T, T> V;
        const int4 *src = reinterpret_cast<const int4 *>(&A);
        int4 *dst = reinterpret_cast<int4 *>(&V);
        for (int e = threadIdx.x; e < (int)(sizeof(V) / sizeof(int4)); e += blockDim.x) dst[e] = src[e];
        __syncthreads();
        if (threadIdx.x == 0) {
            V.nodal = A.nodal_t;
            V.psi = A.psi_t;
            V.slopes = nullptr;
        }
        __syncthreads();
        return &V;
    }
};
template <typename T>
struct TrView<T, T> {
    __device__ static const Args<T, T> *get(const Args<T, T> &A) { return &A; }
};

// Stats and the recycled-basis metadata for the next time step (CTA 0).
// The solution into its optional second destination (fewha_solve_opts.c_out,
// e.g. page-locked host memory): CTA `rank` of `nranks` writes its element
// range once c is final (after the last barrier of the time step, or in a
// launch of its own).
template <typename T, typename S>
__device__ __forceinline__ void phase_store_c(const Args<T, S> &A, int rank, int nranks)
{
    constexpr int W = VW<T>::W;
    long lo, hi;
    cta_range_vec(A.geo.n, W, rank, nranks, lo, hi);
    for (long e = lo + (long)threadIdx.x * W; e < hi; e += (long)blockDim.x * W) {
        T x[W];
        vld_cg(A.c + e, x);
        vst(A.c_out + e, x);
    }
}

template <typename T, typename S>
__device__ __forceinline__ void phase_finish(const Args<T, S> &A, const Basis &b, int K, Scal &sc)
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
