// Solver phases of one reconstructor time step (Ramlau & Stadler,
// Algorithm 3 right-hand side and residual steps, then Algorithm 1 / 2).
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

constexpr int kRedBB = kK * kK + 2 * kK + 12;  // slot of ||b||^2 in Scal::red
constexpr int kRedSize = kK * kK + 2 * kK + 16;

// Shared scalars of a phase (every CTA derives them from the same partials).
struct Scal {
    double red[kRedSize];              // reduced partials
    double tau[kK];                    // projection coefficients
    double chol[kK * kK];              // Cholesky workspace
    double rz, rz_prev, beta, mu, rr, bb, pq, alpha;
    int stop;
};

// Reduced Gram matrix of the old basis (kv x kv) into red[0..kv*kv) .
template <typename T, typename S>
__device__ void reduce_gram(const Args<T, S> &A, int kv, double *out)
{
    for (int i = 0; i < kv; i++) reduce_slots(A.part, A.ncta, kSlotGram + i * kK, kv, out + i * kv);
}

// rz_k of iteration k >= 1 and, if augmented, the projection of z_k
// (Algorithm 2: mu = (z, q_m)/(p_m, q_m), z <- z - mu p_m; or against all).
// Fills sc.rz, sc.mu / sc.tau, sc.rr.
template <typename T, typename S>
__device__ bool iter_scalars(const Args<T, S> &A, const Basis &b, int k, Scal &sc)
{
    const int e0 = kSlotE + ((k - 1) & 1) * kSlotEStride;
    const int kv = b.kv;
    reduce_slots(A.part, A.ncta, e0, 4, sc.red);  // rz, zq, rp, rr
    bool ok = true;
    if (A.recycle_all && kv > 0) {
        reduce_gram(A, kv, sc.red + 8);
        reduce_slots(A.part, A.ncta, e0 + 4, kv, sc.red + 8 + kv * kv);           // Q^T z
        reduce_slots(A.part, A.ncta, e0 + 4 + kK, kv, sc.red + 8 + kv * kv + kv);  // P^T r
    }
    if (threadIdx.x == 0) {
        double rz = sc.red[0];
        sc.mu = 0.0;
        if (kv > 0) {
            if (A.recycle_all) {
                if (!chol_solve(kv, sc.red + 8, sc.red + 8 + kv * kv, sc.tau, sc.chol)) ok = false;
                for (int j = 0; j < kv; j++) rz -= sc.tau[j] * sc.red[8 + kv * kv + kv + j];
            } else {
                double pqm = ldcgd(A.pq + b.ob * A.kcap + b.head);
                sc.mu = sc.red[1] / pqm;
                rz -= sc.mu * sc.red[2];
            }
        }
        sc.rz = rz;
        sc.rr = sc.red[3];
        sc.stop = ok ? 0 : 1;
    }
    __syncthreads();
    return sc.stop == 0;
}

// ---------------------------------------------------------------------------
// R3: right-hand side b = W^{-T} u / delta (u = P^T Gamma^T C s from the
// preceding phases) and the warm-restart residual of Algorithm 3,
// r0 = (b - b_prev) + r_prev;  b_prev <- b.
// ---------------------------------------------------------------------------
template <typename T, typename S>
__device__ void phase_rhs_fdwt(const Args<T, S> &A, T *sm, double *sred)
{
    typedef typename AccT<T>::type Acc;
    Acc acc[2] = {0, 0};
    layer_fdwt<T, S>(A, sm, [&](long e, T b) {
        T r0 = (b - A.b_prev[e]) + ldcg(A.r + e);
        A.b_prev[e] = b;
        A.r[e] = r0;
        acc[0] += (Acc)b * (Acc)b;
        acc[1] += (Acc)r0 * (Acc)r0;
    });
    const int slots[2] = {kSlotR2, kSlotR2 + 1};
    block_partials<2>(acc, A.part, slots, sred);
}

// Gram matrix (p_i, q_j) of the old basis and P^T r0 (Algorithm 2 init).
template <typename T, typename S>
__device__ void phase_gram(const Args<T, S> &A, const Basis &b)
{
    long lo, hi;
    cta_range(A.geo.n, lo, hi);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int kv = b.kv, ns = kv * kv + kv;
    for (int s = warp; s < ns; s += nw) {
        const T *X, *Y;
        int slot;
        if (s < kv * kv) {
            X = oldQ(A, b, s % kv);
            Y = oldP(A, b, s / kv);
            slot = kSlotGram + (s / kv) * kK + (s % kv);
        } else {
            X = oldP(A, b, s - kv * kv);
            Y = A.r;  // written by another CTA in R3
            slot = kSlotGram + kK * kK + (s - kv * kv);
        }
        typename AccT<T>::type acc = 0;
        for (long e = lo + lane; e < hi; e += 32) acc += __ldg(X + e) * ldcg(Y + e);
        acc = warp_sum_t(acc);
        if (lane == 0) A.part[(size_t)slot * kMaxCtas + blockIdx.x] = (double)acc;
    }
}

// c += P sigma, r -= Q sigma with sigma = G^{-1} P^T r0; then (q_j, z), (r, z), (r, r).
template <typename T, typename S>
__device__ bool phase_init(const Args<T, S> &A, const Basis &b, Scal &sc)
{
    const int kv = b.kv;
    reduce_gram(A, kv, sc.red);
    reduce_slots(A.part, A.ncta, kSlotGram + kK * kK, kv, sc.red + kv * kv);
    if (threadIdx.x == 0) {
        sc.stop = chol_solve(kv, sc.red, sc.red + kv * kv, sc.tau, sc.chol) ? 0 : 1;
        if (sc.stop) set_status(A.rec, FEWHA_ERR_NOT_SPD);
    }
    __syncthreads();
    if (sc.stop) return false;
    long lo, hi;
    cta_range(A.geo.n, lo, hi);
    for (long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
        T cv = A.c[e], rv = ldcg(A.r + e);
        for (int j = 0; j < kv; j++) {
            const T sj = (T)sc.tau[j];
            cv += sj * __ldg(oldP(A, b, j) + e);
            rv -= sj * __ldg(oldQ(A, b, j) + e);
        }
        A.c[e] = cv;
        A.r[e] = rv;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = warp; s < kv + 2; s += nw) {
        typename AccT<T>::type acc = 0;
        for (long e = lo + lane; e < hi; e += 32) {
            const T rv = ldcg(A.r + e), z = __ldg(A.geo.invJ + e) * rv;
            if (s < kv)
                acc += __ldg(oldQ(A, b, s) + e) * z;
            else if (s == kv)
                acc += rv * z;
            else
                acc += rv * rv;
        }
        acc = warp_sum_t(acc);
        int slot = s < kv ? kSlotInit + s : (s == kv ? kSlotInit + kK : kSlotInit + kK + 1);
        if (lane == 0) A.part[(size_t)slot * kMaxCtas + blockIdx.x] = (double)acc;
    }
    return true;
}

// ---------------------------------------------------------------------------
// A_k: direction update fused with W^{-1}:
//   k = 0: p_0 = z_0 - P G^{-1} Q^T z_0 (Algorithm 2) or z_0 (Algorithm 1)
//   k > 0: p_k = (z_k - mu p_m) + beta p_{k-1},  beta = rz_k / rz_{k-1}
// Returns false (uniformly) when the stopping test holds before iteration k.
// ---------------------------------------------------------------------------
template <typename T, typename S>
__device__ bool phase_A(const Args<T, S> &A, const Basis &b, int k, T *sm, Scal &sc, double *sred)
{
    const int kv = b.kv;
    if (k == 0) {
        reduce_slots(A.part, A.ncta, kSlotR2, 2, sc.red);
        if (kv > 0) {
            reduce_slots(A.part, A.ncta, kSlotInit, kv, sc.red + 2);
            reduce_slots(A.part, A.ncta, kSlotInit + kK + 1, 1, sc.red + 2 + kv);
            reduce_gram(A, kv, sc.red + 8 + kK);
        }
        if (threadIdx.x == 0) {
            sc.bb = sc.red[0];
            sc.rr = kv > 0 ? sc.red[2 + kv] : sc.red[1];
            sc.stop = 0;
            if (kv > 0 && !chol_solve(kv, sc.red + 8 + kK, sc.red + 2, sc.tau, sc.chol)) {
                sc.stop = 1;
                set_status(A.rec, FEWHA_ERR_NOT_SPD);
            }
            sc.beta = 0.0;
            sc.mu = 0.0;
        }
        __syncthreads();
        if (sc.stop) return false;
    } else {
        reduce_slots(A.part, A.ncta, kSlotR2, 1, sc.red + kRedBB);
        if (!iter_scalars(A, b, k, sc)) {
            if (threadIdx.x == 0) set_status(A.rec, FEWHA_ERR_NOT_SPD);
            return false;
        }
        if (threadIdx.x == 0) {
            sc.bb = sc.red[kRedBB];
            sc.rz_prev = ldcgd(A.rec->rz + (k - 1));
            sc.beta = sc.rz / sc.rz_prev;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sc.stop = (A.rtol > 0.0 && sc.rr <= A.rtol * A.rtol * sc.bb) ? 1 : 0;
        if (sc.stop && blockIdx.x == 0) {
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
    T tau[kK];
    for (int j = 0; j < kK; j++) tau[j] = j < kv ? (T)sc.tau[j] : T(0);
    const bool proj_all = (k == 0) || A.recycle_all;
    typedef typename AccT<T>::type Acc;
    Acc acc[2] = {0, 0};
    layer_idwt<T, S>(A, sm, [&](long e) -> T {
        const T rv = ldcg(A.r + e);
        T z = __ldg(A.geo.invJ + e) * rv;
        if (kv > 0) {
            if (proj_all) {
                for (int j = 0; j < kv; j++) z -= tau[j] * __ldg(oldP(A, b, j) + e);
            } else {
                z -= mu * __ldg(pm + e);
            }
        }
        const T p = k > 0 ? z + beta * pprev[e] : z;
        pk[e] = p;
        acc[0] += (Acc)__ldg(A.geo.alpha_d + e) * (Acc)p * (Acc)p;
        acc[1] += (Acc)rv * (Acc)p;
        return p;
    });
    const int slots[2] = {kSlotA + (k & 1) * 2, kSlotA + (k & 1) * 2 + 1};
    block_partials<2>(acc, A.part, slots, sred);
    return true;
}

// rz_k as seen by CD_k and E_k (identical arithmetic to phase_A).
template <typename T, typename S>
__device__ bool rz_of_iter(const Args<T, S> &A, const Basis &b, int k, Scal &sc)
{
    if (k == 0) {
        reduce_slots(A.part, A.ncta, kSlotA + 1, 1, sc.red);
        if (threadIdx.x == 0) sc.rz = sc.red[0];
        __syncthreads();
        return true;
    }
    return iter_scalars(A, b, k, sc);
}

// ---------------------------------------------------------------------------
// C_k: scalars of iteration k and u = P^T psi.  (p_k, q_k) comes from the
// forward pass: sum w s^2 (WFS phase) + sum alpha d p^2 (A phase), equal to
// (p_k, M p_k) by Eq. M.  Returns false (uniformly) on rz == 0 (converged)
// or breakdown; CTA 0 records rz_k, alpha_k and (p_k, q_k).
// ---------------------------------------------------------------------------
template <typename T, typename S>
__device__ bool phase_C(const Args<T, S> &A, const Basis &b, int k, T *sm, Scal &sc)
{
    if (!rz_of_iter(A, b, k, sc)) return false;
    reduce_slots(A.part, A.ncta, kSlotB + (k & 1), 1, sc.red + 1);
    reduce_slots(A.part, A.ncta, kSlotA + (k & 1) * 2, 1, sc.red + 2);
    if (threadIdx.x == 0) {
        sc.pq = sc.red[1] + sc.red[2];
        sc.stop = 0;
        if (sc.rz == 0.0) {
            sc.stop = 1;
        } else if (!(sc.pq > 0.0) || !isfinite(sc.pq) || !isfinite(sc.rz)) {
            sc.stop = 1;
            if (blockIdx.x == 0) set_status(A.rec, FEWHA_ERR_BREAKDOWN);
        }
        sc.alpha = sc.rz / sc.pq;
        if (blockIdx.x == 0) {
            if (sc.stop) {
                A.rec->iters = k;
                A.rec->done = 1;
            } else {
                A.rec->rz[k] = sc.rz;
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

// D_k: q_k = W^{-T} u / delta + alpha D p_k, stored in the basis slot.
template <typename T, typename S>
__device__ void phase_D(const Args<T, S> &A, const Basis &b, int k, T *sm)
{
    const T *pk = newP(A, b, k);
    T *qk = newQ(A, b, k);
    layer_fdwt<T, S>(A, sm, [&](long e, T v) { qk[e] = v + __ldg(A.geo.alpha_d + e) * pk[e]; });
}

// E_k: c += alpha p, r -= alpha q, and the inner products of the next step.
template <typename T, typename S>
__device__ void phase_E(const Args<T, S> &A, const Basis &b, int k, double *sred)
{
    const T alpha = (T)ldcgd(A.rec->alpha + k);
    const T *pk = newP(A, b, k), *qk = newQ(A, b, k);
    const int kv = b.kv;
    const T *pm = kv > 0 ? oldP(A, b, kv - 1) : nullptr;
    const T *qm = kv > 0 ? oldQ(A, b, kv - 1) : nullptr;
    long lo, hi;
    cta_range(A.geo.n, lo, hi);
    typedef typename AccT<T>::type Acc;
    Acc acc[4] = {0, 0, 0, 0};
    for (long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
        const T p = ldcg(pk + e), q = ldcg(qk + e);
        const T cv = A.c[e] + alpha * p;
        const T rv = ldcg(A.r + e) - alpha * q;
        A.c[e] = cv;
        A.r[e] = rv;
        const T z = __ldg(A.geo.invJ + e) * rv;
        acc[0] += (Acc)rv * (Acc)z;
        if (kv > 0 && !A.recycle_all) {
            acc[1] += (Acc)z * (Acc)__ldg(qm + e);
            acc[2] += (Acc)rv * (Acc)__ldg(pm + e);
        }
        acc[3] += (Acc)rv * (Acc)rv;
    }
    const int e0 = kSlotE + (k & 1) * kSlotEStride;
    const int slots[4] = {e0, e0 + 1, e0 + 2, e0 + 3};
    block_partials<4>(acc, A.part, slots, sred);
    if (kv > 0 && A.recycle_all) {
        __syncthreads();
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int s = warp; s < 2 * kv; s += nw) {
            Acc a = 0;
            for (long e = lo + lane; e < hi; e += 32) {
                const T rv = ldcg(A.r + e);
                if (s < kv)
                    a += (Acc)(__ldg(A.geo.invJ + e) * rv) * (Acc)__ldg(oldQ(A, b, s) + e);
                else
                    a += (Acc)rv * (Acc)__ldg(oldP(A, b, s - kv) + e);
            }
            a = warp_sum_t(a);
            int slot = s < kv ? e0 + 4 + s : e0 + 4 + kK + (s - kv);
            if (lane == 0) A.part[(size_t)slot * kMaxCtas + blockIdx.x] = (double)a;
        }
    }
}

// Stats and the recycled-basis metadata for the next time step (CTA 0).
template <typename T, typename S>
__device__ void phase_finish(const Args<T, S> &A, const Basis &b, int K, Scal &sc)
{
    const int e0 = kSlotE + ((K - 1) & 1) * kSlotEStride;
    reduce_slots(A.part, A.ncta, kSlotR2, 2, sc.red);
    if (K > 0)
        reduce_slots(A.part, A.ncta, e0, 4, sc.red + 2);
    else if (b.kv > 0)
        reduce_slots(A.part, A.ncta, kSlotInit + kK, 2, sc.red + 2 + 2);
    if (threadIdx.x == 0) {
        double bb = sc.red[0];
        double rr = K > 0 ? sc.red[2 + 3] : (b.kv > 0 ? sc.red[2 + 3] : sc.red[1]);
        double rz = K > 0 ? sc.red[2] : (b.kv > 0 ? sc.red[2 + 2] : 0.0);
        fewha_stats st;
        st.status = ldcgi(&A.rec->status);
        st.iterations = K;
        st.bnorm = sqrt(bb);
        st.rel_res = bb > 0 ? sqrt(rr / bb) : 0.0;
        st.rz = rz;
        int count = ldcgi(A.meta + 1);
        if (K > 0) {
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
