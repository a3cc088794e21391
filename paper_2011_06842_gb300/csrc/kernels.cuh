// Kernels of the FEWHA hot path and the per-precision implementation
// object that launches them (internal to libfewha).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <cstddef>
#include <cstring>
#include <type_traits>
#include <vector>

#include "mcao.cuh"
#include "plan.h"
#include "solver.cuh"

namespace fewha {

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T *dyn_smem()
{
    extern __shared__ __align__(16) unsigned char fewha_smem[];
    return reinterpret_cast<T *>(fewha_smem);
}

// Kernel arguments are copied into shared memory once: the phases are not
// inlined and take them by reference, which would otherwise place them in
// local memory (a load through the L1 for every field read).
template <typename T, typename S>
__device__ __forceinline__ void args_to_smem(const Args<T, S> &src, Args<T, S> &dst)
{
    const int4 *s = reinterpret_cast<const int4 *>(&src);
    int4 *d = reinterpret_cast<int4 *>(&dst);
    for (int e = threadIdx.x; e < (int)(sizeof(Args<T, S>) / sizeof(int4)); e += blockDim.x) d[e] = s[e];
    __syncthreads();
}

// apply: nodal = W^{-1} x
template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_apply_idwt(const __grid_constant__ Args<T, S> Ap)
{
    __shared__ __align__(16) Args<T, S> A;
    args_to_smem(Ap, A);
    constexpr int W = VW<T>::W;
    layer_idwt<T, S>(A, dyn_smem<T>(), [&](long e, T (&x)[W]) { vld(A.x + e, x); });
}

// psi = Gamma^T C Gamma P nodal (RHS = false) or Gamma^T C s (RHS = true)
template <typename T, typename S, bool RHS>
__global__ void __launch_bounds__(kThreads, 1) k_wfs(const __grid_constant__ Args<T, S> Ap)
{
    __shared__ __align__(16) Args<T, S> A;
    args_to_smem(Ap, A);
    __shared__ double sred[kSred];
    typename AccT<T>::type acc[1] = {wfs_phase<T, S, RHS>(A, dyn_smem<T>())};
    const int slots[1] = {kSlotB};
    block_partials<1>(acc, A.part, slots, sred, A.vrank());
}

// u = P^T psi
template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_gather(const __grid_constant__ Args<T, S> Ap)
{
    __shared__ __align__(16) Args<T, S> A;
    args_to_smem(Ap, A);
    if (ldcgi(&A.rec->done) || ldcgi(&A.rec->status)) return;
    band_gather<T, S>(A, dyn_smem<T>());
}

// y = W^{-T} u + alpha D x  (APPLY) or y = W^{-T} u (RHS)
template <typename T, typename S, bool RHS>
__global__ void __launch_bounds__(kThreads, 1) k_fdwt(const __grid_constant__ Args<T, S> Ap)
{
    __shared__ __align__(16) Args<T, S> A;
    args_to_smem(Ap, A);
    constexpr int W = VW<T>::W;
    layer_fdwt<T, S>(A, dyn_smem<T>(), [&](long e, const T (&v)[W]) {
        T y[W], x[W], ad[W];
        if (!RHS) {
            vld(A.x + e, x);
            vld_nc(A.geo.alpha_d + e, ad);
        }
#pragma unroll
        for (int i = 0; i < W; i++) y[i] = RHS ? v[i] : v[i] + ad[i] * x[i];
        vst(A.y + e, y);
    });
}

// --- y_v = M x_v for several vectors at once --------------------------------
// Vector v is applied by CTAs [v*per, (v+1)*per) with its own scratch
// buffers, so the per-layer transforms of all vectors run side by side.
constexpr int kMaxVec = FEWHA_MAX_MULTI;

template <typename T, typename S>
struct MultiArgs {
    Args<T, S> a[kMaxVec];
    int per;
};

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_multi_idwt(const __grid_constant__ MultiArgs<T, S> M)
{
    __shared__ __align__(16) Args<T, S> A;
    args_to_smem(M.a[blockIdx.x / M.per], A);
    constexpr int W = VW<T>::W;
    layer_idwt<T, S>(A, dyn_smem<T>(), [&](long e, T (&x)[W]) { vld(A.x + e, x); });
}

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_multi_wfs(const __grid_constant__ MultiArgs<T, S> M)
{
    __shared__ __align__(16) Args<T, S> A;
    args_to_smem(M.a[blockIdx.x / M.per], A);
    __shared__ double sred[kSred];
    typename AccT<T>::type acc[1] = {wfs_phase<T, S, false>(A, dyn_smem<T>())};
    const int slots[1] = {kSlotB};
    block_partials<1>(acc, A.part, slots, sred, A.vrank());
}

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_multi_gather(const __grid_constant__ MultiArgs<T, S> M)
{
    __shared__ __align__(16) Args<T, S> A;
    args_to_smem(M.a[blockIdx.x / M.per], A);
    band_gather<T, S>(A, dyn_smem<T>());
}

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_multi_fdwt(const __grid_constant__ MultiArgs<T, S> M)
{
    __shared__ __align__(16) Args<T, S> A;
    args_to_smem(M.a[blockIdx.x / M.per], A);
    constexpr int W = VW<T>::W;
    layer_fdwt<T, S>(A, dyn_smem<T>(), [&](long e, const T (&v)[W]) {
        T y[W], x[W], ad[W];
        vld(A.x + e, x);
        vld_nc(A.geo.alpha_d + e, ad);
#pragma unroll
        for (int i = 0; i < W; i++) y[i] = v[i] + ad[i] * x[i];
        vst(A.y + e, y);
    });
}

// --- mirror side of the reconstructor loop (Algorithm 3) --------------------
// One deformable mirror conjugated to the ground with its actuators on the
// (n_s+1)^2 pupil nodes (reading of the fitting operator F).
template <typename T>
struct FitTab {
    long off[FEWHA_MAX_LAYERS];
    int n[FEWHA_MAX_LAYERS];
    int L, m;
    const int *fk;  // [L][m] lower node of pupil index j (both axes)
    const T *fw;    // [L][m] fractional position
};

// a~ = F W^{-1} c with nodal = W^{-1} c already in place: on-axis bilinear
// sample of every layer at every actuator, summed over layers.
template <typename T, typename S>
__global__ void k_fit(const __grid_constant__ FitTab<T> F, const S *__restrict__ nodal, T *__restrict__ a)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= F.m * F.m) return;
    const int i = e / F.m, j = e - i * F.m;
    T v = 0;
    for (int l = 0; l < F.L; l++) {
        const int n = F.n[l];
        const int kx = F.fk[l * F.m + j], ky = F.fk[l * F.m + i];
        const T wx = F.fw[l * F.m + j], wy = F.fw[l * F.m + i];
        const S *Lp = nodal + F.off[l] + (long)ky * n + kx;
        const T v00 = Cv<S>::ld(Lp[0]), v01 = Cv<S>::ld(Lp[1]);
        const T v10 = Cv<S>::ld(Lp[n]), v11 = Cv<S>::ld(Lp[n + 1]);
        v += (T(1) - wy) * ((T(1) - wx) * v00 + wx * v01) + wy * ((T(1) - wx) * v10 + wx * v11);
    }
    a[e] = v;
}

// Pseudo-open-loop slopes: s_out = s + Gamma a for every guide star (the
// ground mirror adds the same phase to every sensor).
template <typename T, typename S>
__global__ void k_pol(const S *s_in, const T *__restrict__ a, S *s_out, int G, int ns)  // s_out may be s_in
{
    const int m = ns + 1, per = ns * ns;
    const long total = (long)G * per;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int g = (int)(idx / per), e = (int)(idx - (long)g * per);
        const int i = e / ns, j = e - i * ns;
        const T p00 = a[i * m + j], p01 = a[i * m + j + 1];
        const T p10 = a[(i + 1) * m + j], p11 = a[(i + 1) * m + j + 1];
        const T gx = T(0.5) * ((p01 - p00) + (p11 - p10));
        const T gy = T(0.5) * ((p10 - p00) + (p11 - p01));
        const size_t b = (size_t)g * 2 * per;
        s_out[b + e] = Cv<S>::st(Cv<S>::ld(s_in[b + e]) + gx);
        s_out[b + per + e] = Cv<S>::st(Cv<S>::ld(s_in[b + per + e]) + gy);
    }
}

// Gain control: closed loop a_next = a_i + gain (a~ - a_{i-1}); open loop
// a_next = (1 - gain) a_i + gain a~.
template <typename T>
__global__ void k_control(int closed, T gain, const T *__restrict__ am1, const T *__restrict__ ai,
                          const T *__restrict__ af, T *__restrict__ an, int na)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < na; e += gridDim.x * blockDim.x)
        an[e] = closed ? ai[e] + gain * (af[e] - am1[e]) : (T(1) - gain) * ai[e] + gain * af[e];
}

// --- solver phases, one kernel each (FEWHA_LAUNCH_PHASES) -------------------
#define FEWHA_PHASE_GUARD                                             \
    __shared__ Scal sc;                                               \
    __shared__ double sred[kSred];                                   \
    __shared__ __align__(16) Args<T, S> A;                            \
    args_to_smem(Ap, A);                                              \
    (void)sred;                                                       \
    if (ldcgi(&A.rec->done) || ldcgi(&A.rec->status)) return;         \
    const Basis b = basis_info(A);                                    \
    (void)b;

// R1: weighted slopes -> psi, and the Gram matrix of the old basis
template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_rhs_wfs(const __grid_constant__ Args<T, S> Ap)
{
    __shared__ __align__(16) Args<T, S> A;
    args_to_smem(Ap, A);
    if (!A.rhs_in_state) wfs_phase<T, S, true>(A, dyn_smem<T>());
    const Basis b = basis_info(A);
    if (b.kv > 0) phase_gram<T, S>(A, b, dyn_smem<T>(), (int)(A.smem_bytes / sizeof(T)));
}

// R2: u = P^T psi; the last CTA also factorises the Gram matrix
template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_rhs_gather(const __grid_constant__ Args<T, S> Ap)
{
    FEWHA_PHASE_GUARD
    if (!A.rhs_in_state) band_gather<T, S>(A, dyn_smem<T>());
    if (b.kv > 0 && A.vrank() == A.ncta - 1) phase_factor<T, S>(A, b, sc);
}

// R3: the finest analysis level of u (split form), then b, r0 and P^T r0
template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_rhs_D1(const __grid_constant__ Args<T, S> Ap)
{
    FEWHA_PHASE_GUARD
    (void)sc;
    if (!A.rhs_in_state) phase_D1<T, S>(A, dyn_smem<T>());
}

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_rhs_update(const __grid_constant__ Args<T, S> Ap)
{
    FEWHA_PHASE_GUARD
    (void)sc;
    if (A.rhs_in_state)
        phase_rhs_update<T, S, true>(A, b, dyn_smem<T>(), sred);
    else
        phase_rhs_update<T, S, false>(A, b, dyn_smem<T>(), sred);
}

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_init(const __grid_constant__ Args<T, S> Ap)
{
    FEWHA_PHASE_GUARD
    if (b.kv > 0) phase_init<T, S>(A, b, sc, sred);
}

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_UA1(const __grid_constant__ Args<T, S> Ap, int k)
{
    FEWHA_PHASE_GUARD
    phase_UA1<T, S>(A, b, k, dyn_smem<T>(), sc, sred);
}

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_A2(const __grid_constant__ Args<T, S> Ap, int k)
{
    FEWHA_PHASE_GUARD
    (void)sc;
    phase_A2<T, S>(A, b, k, dyn_smem<T>());
}

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_B(const __grid_constant__ Args<T, S> Ap, int k)
{
    FEWHA_PHASE_GUARD
    (void)sc;
    typename AccT<T>::type acc[1] = {wfs_phase<T, S, false>(A, dyn_smem<T>())};
    const int slots[1] = {kSlotB + (k & 1)};
    block_partials<1>(acc, A.part, slots, sred, A.vrank());
}

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_C(const __grid_constant__ Args<T, S> Ap, int k)
{
    FEWHA_PHASE_GUARD
    phase_C<T, S>(A, b, k, dyn_smem<T>(), sc);
}

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_D1(const __grid_constant__ Args<T, S> Ap, int k)
{
    FEWHA_PHASE_GUARD
    (void)sc;
    phase_D1<T, S>(A, dyn_smem<T>());
}

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_D2E(const __grid_constant__ Args<T, S> Ap, int k)
{
    FEWHA_PHASE_GUARD
    (void)sc;
    phase_D2E<T, S>(A, b, k, dyn_smem<T>(), sred);
}

// residual replacement after iteration k (phases TU, TA2, TB, TC, TD1, TE)
template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_TU(const __grid_constant__ Args<T, S> Ap)
{
    FEWHA_PHASE_GUARD
    (void)sc;
    phase_TU<T>(*TrView<T, S>::get(A), dyn_smem<T>());
}

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_TA2(const __grid_constant__ Args<T, S> Ap)
{
    FEWHA_PHASE_GUARD
    (void)sc;
    const Args<T, T> &V = *TrView<T, S>::get(A);
    phase_fine_synth<T, T>(V, V.c, dyn_smem<T>());
}

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_TB(const __grid_constant__ Args<T, S> Ap)
{
    FEWHA_PHASE_GUARD
    (void)sc;
    wfs_phase<T, T, false>(*TrView<T, S>::get(A), dyn_smem<T>());
}

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_TC(const __grid_constant__ Args<T, S> Ap)
{
    FEWHA_PHASE_GUARD
    (void)sc;
    band_gather<T, T>(*TrView<T, S>::get(A), dyn_smem<T>());
}

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_TD1(const __grid_constant__ Args<T, S> Ap)
{
    FEWHA_PHASE_GUARD
    (void)sc;
    phase_D1<T, T>(*TrView<T, S>::get(A), dyn_smem<T>());
}

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_TE(const __grid_constant__ Args<T, S> Ap, int k)
{
    FEWHA_PHASE_GUARD
    (void)sc;
    phase_TE<T>(*TrView<T, S>::get(A), b, k, dyn_smem<T>(), sred);
}

template <typename T, typename S>
__global__ void __launch_bounds__(kThreads, 1) k_finish(const __grid_constant__ Args<T, S> Ap)
{
    __shared__ Scal sc;
    __shared__ __align__(16) Args<T, S> A;
    args_to_smem(Ap, A);
    if (A.c_out) phase_store_c<T, S>(A, blockIdx.x, gridDim.x);  // this launch's CTAs
    if (A.vrank() != 0) return;
    const Basis b = basis_info(A);
    int K = ldcgi(&A.rec->done) ? ldcgi(&A.rec->iters) : A.max_iter;
    phase_finish<T, S>(A, b, K, sc);
}

// Residual replacement after iteration k inside the persistent kernel (phases
// TU, TA2, TB, TC, TD1, TE, each followed by the group's barrier); false when a
// barrier reports an error.  ti: trace slot of the next barrier.
template <typename T>
__device__ __forceinline__ bool true_residual_phases(const Args<T, T> &V, const Basis &b, int k, double *sred,
                                                     int rank, int &ti)
{
    T *sm = dyn_smem<T>();
    const bool split = split_levels(V);
    auto sync = [&](int tag) -> bool {
        unsigned long long *slot = (V.trace && ti < V.trace_cap) ? V.trace + 4 * ti : nullptr;
        if (slot && rank == 0 && threadIdx.x == 0) slot[3] = (unsigned long long)tag;
        ti++;
        return grid_sync(V.rec, V.timeout_ns, V.ncta, rank, slot);
    };
    phase_TU<T>(V, sm);
    if (!sync(20)) return false;
    if (split) {
        phase_fine_synth<T, T>(V, V.c, sm);
        if (!sync(21)) return false;
    }
    wfs_phase<T, T, false>(V, sm);
    if (!sync(22)) return false;
    band_gather<T, T>(V, sm);
    if (!sync(23)) return false;
    if (split) {
        phase_D1<T, T>(V, sm);
        if (!sync(24)) return false;
    }
    phase_TE<T>(V, b, k, sm, sred);
    return sync(25);
}

// --- the whole time step of one instance, run by its group of CTAs ----------
// TR: the kernel variant with the residual replacement (fewha_solve_opts.
// true_res_every > 0); RIS: the variant for a right-hand side already in the
// state (fewha_solve_opts.rhs_in_state).  The default variant carries the
// code of neither, so its register allocation does not depend on them.
template <typename T, typename S, bool TR, bool RIS = false>
__device__ void solve_body(const Args<T, S> &A, Scal &sc, double *sred)
{
    T *sm = dyn_smem<T>();
    const unsigned long long to = A.timeout_ns;
    const Basis b = basis_info(A);
    const int rank = A.vrank();
    int ti = 0;  // trace slot of the next barrier
    // barrier of the group with the optional phase trace (tag = phase id)
    auto sync = [&](int tag) -> bool {
        unsigned long long *slot = (A.trace && ti < A.trace_cap) ? A.trace + 4 * ti : nullptr;
        if (slot && rank == 0 && threadIdx.x == 0) slot[3] = (unsigned long long)tag;
        bool ok = grid_sync(A.rec, to, A.ncta, rank, slot);
        ti++;
        return ok;
    };
    int K = A.max_iter;
    const bool split = split_levels(A);  // uniform over the instance's CTAs
    const Args<T, T> *V = nullptr;  // residual replacement's view of the arguments
    if constexpr (TR) V = TrView<T, S>::get(A);
    trace_begin(A.trace != nullptr);
    constexpr bool rhs = !RIS;  // form the right-hand side (else it is in the state)
    do {
        if (rhs) wfs_phase<T, S, true>(A, sm);
        if (b.kv > 0) phase_gram<T, S>(A, b, sm, (int)(A.smem_bytes / sizeof(T)));
        if ((rhs || b.kv > 0) && !sync(1)) break;
        if (rhs) band_gather<T, S>(A, sm);
        if (b.kv > 0 && rank == A.ncta - 1) phase_factor<T, S>(A, b, sc);
        if ((rhs || b.kv > 0) && !sync(2)) break;
        if (split && rhs) {
            phase_D1<T, S>(A, sm);  // the finest analysis level of u
            if (!sync(6)) break;
        }
        phase_rhs_update<T, S, RIS>(A, b, sm, sred);  // b, r0 and P^T r0
        if (!sync(3)) break;
        if (b.kv > 0) {
            phase_init<T, S>(A, b, sc, sred);
            if (!sync(5)) break;
        }
        for (int k = 0; k < A.max_iter; k++) {
            // UA1's partial sums join the WFS phase's block reduction
            typename AccT<T>::type ua[2];
            if (!phase_UA1<T, S>(A, b, k, sm, sc, sred, true, ua)) {
                K = k;
                break;
            }
            if (!sync(10)) break;
            if (split) {
                phase_A2<T, S>(A, b, k, sm);
                if (!sync(16)) break;
            }
            {
                typename AccT<T>::type acc[3] = {wfs_phase<T, S, false>(A, sm), ua[0], ua[1]};
                const int slots[3] = {kSlotB + (k & 1), kSlotA + (k & 1) * 2, kSlotA + (k & 1) * 2 + 1};
                block_partials<3>(acc, A.part, slots, sred, rank);
            }
            if (!sync(12)) break;
            if (!phase_C<T, S>(A, b, k, sm, sc, true)) {
                K = k;
                break;
            }
            if (!sync(13)) break;
            if (split) {
                phase_D1<T, S>(A, sm);
                if (!sync(14)) break;
            }
            phase_D2E<T, S>(A, b, k, sm, sred, &sc.alpha);
            if (!sync(15)) break;
            // residual replacement: r = b - M c, then iteration k+1's scalars
            // come from it
            if constexpr (TR) {
                if ((k + 1) % A.true_res_every == 0 && !true_residual_phases<T>(*V, b, k, sred, rank, ti)) break;
            }
        }
    } while (0);
    // on a device-side error the stats carry the status; the other fields are
    // then not meaningful
    if (A.c_out) phase_store_c<T, S>(A, rank, A.ncta);
    if (rank == 0) phase_finish<T, S>(A, b, K, sc);
}

// One instance on the whole grid (cooperative launch).
template <typename T, typename S, bool TR, bool RIS = false>
__global__ void __launch_bounds__(kThreads, 1) k_solve_persistent(const __grid_constant__ Args<T, S> Ap)
{
    __shared__ Scal sc;
    __shared__ double sred[kSred];
    __shared__ __align__(16) Args<T, S> A;
    args_to_smem(Ap, A);
    solve_body<T, S, TR, RIS>(A, sc, sred);
}

// Many instances in one cooperative launch: CTA c runs instance cta_inst[c]
// with the group of CTAs [inst.cta0, inst.cta0 + inst.ncta).
template <typename T, typename S, bool TR>
__global__ void __launch_bounds__(kThreads, 1) k_solve_batched(const Args<T, S> *inst, const int *cta_inst,
                                                              int nrounds, int total, Record *brec,
                                                              unsigned long long timeout_ns)
{
    // Instances run in rounds: in round r, CTA c runs instance cta_inst[r * total + c]
    // (-1: idle in this round); a barrier over the whole launch separates rounds, so
    // one launch can give a few large instances many CTAs and then the small ones.
    __shared__ Scal sc;
    __shared__ double sred[kSred];
    __shared__ __align__(16) Args<T, S> A;
    for (int r = 0; r < nrounds; r++) {
        const int i = cta_inst[r * total + blockIdx.x];
        if (i >= 0) {
            args_to_smem(inst[i], A);
            solve_body<T, S, TR>(A, sc, sred);
        }
        if (r + 1 < nrounds && !grid_sync(brec, timeout_ns, total, blockIdx.x)) return;
    }
}

// Resets the record flags and the barrier of every instance of a batch.
template <typename T, typename S>
__global__ void k_batch_reset(const Args<T, S> *inst, int n, Record *brec)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        brec->status = 0;
        brec->bar.count = brec->bar.gen = 0;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        Record *r = inst[i].rec;
        r->status = r->done = r->iters = r->chol_ok = 0;
        r->bar.count = r->bar.gen = 0;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
#define CK(x)                                   \
    do {                                        \
        cudaError_t _e = (x);                   \
        if (_e != cudaSuccess) return FEWHA_ERR_CUDA; \
    } while (0)

template <typename T>
static int upload(const std::vector<T> &v, T **d)
{
    *d = nullptr;
    if (v.empty()) return FEWHA_OK;
    if (cudaMalloc(d, v.size() * sizeof(T)) != cudaSuccess) return FEWHA_ERR_NOMEM;
    CK(cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return FEWHA_OK;
}

struct ImplBase {
    virtual ~ImplBase() {}
    virtual int init(int grid) = 0;
    virtual int get_invJ(double *host) const = 0;
    virtual int apply(const void *x, void *y, cudaStream_t s) = 0;
    // mirror side of Algorithm 3 (ground DM on the pupil nodes)
    virtual int fit(const void *c, void *a, cudaStream_t s) = 0;
    virtual int pol_slopes(const void *s_in, const void *a, void *s_out, cudaStream_t s) = 0;
    virtual int control(int closed, double gain, const void *am1, const void *ai, const void *af, void *an,
                        cudaStream_t s) = 0;
    // MCAO fitting onto several mirrors: plan (tables, work vectors), fit, free
    virtual int mcao_create(const fewha_mcao_desc *d, void **plan, long *n_act) = 0;
    virtual int mcao_fit(void *plan, const void *c, void *a, int iters, cudaStream_t s) = 0;
    virtual void mcao_destroy(void *plan) = 0;
    // y_v = M x_v for v < nvec (x_v = x + v*ldx, y_v = y + v*ldy), nvec <= kMaxVec
    virtual int apply_multi(const void *x, long ldx, void *y, long ldy, int nvec, cudaStream_t s) = 0;
    virtual int rhs(const void *sl, void *b, cudaStream_t s) = 0;
    virtual int solve(const void *sl, void *c, const fewha_state *st, const fewha_solve_opts *o,
                      fewha_stats *stats, cudaStream_t s) = 0;
    virtual int set_invJ(const std::vector<double> &invJ) = 0;
    // C_eta^{-1}: weight of guide star g on its lit subapertures (plan.geom.gs[g].weight)
    virtual int set_weights() = 0;
    virtual void set_trace(unsigned long long *buf, int cap) = 0;
    virtual void set_timeout(unsigned long long ns) = 0;
    // --- batched launch support (many instances, one cooperative kernel) ---
    virtual size_t args_size() const = 0;
    virtual int precision_id() const = 0;
    // WFS tile shape for a group of `ctas` CTAs, and the dynamic shared memory it needs
    virtual int tiles_for(int ctas, int *ty, int *tx) const = 0;
    virtual size_t smem_for(int ty, int tx) const = 0;
    // host copy of this instance's kernel arguments for one time step
    virtual int batch_args(void *out, const void *sl, void *c, const fewha_state *st, const fewha_solve_opts *o,
                           fewha_stats *stats, int cta0, int ncta, int ty, int tx, size_t smem) const = 0;
    // CTAs that can be co-resident for the batched kernel with `smem` bytes
    virtual int batch_capacity(size_t smem, int *max_ctas) const = 0;
    virtual int launch_batched(const void *d_args, const int *d_map, int n, int total, size_t smem, int nrounds,
                               Record *brec, int true_res, cudaStream_t s) const = 0;
    // y = M x with every scratch buffer carved from caller-provided device
    // memory (no allocation); FEWHA_ERR_SCRATCH if `bytes` is too small.
    virtual int apply_in_scratch(const void *x, void *y, void *scratch, size_t bytes, cudaStream_t s) = 0;
    virtual void launch_info(fewha_launch_info *out) const = 0;
    // P^T band heights (layer rows) on the largest and on the smaller layers
    virtual int set_bands(int rows_large, int rows_small) = 0;
};

template <typename T, typename S>
struct Impl : ImplBase {
    const Plan &P;
    Args<T, S> base{};
    int ncta = 1;
    size_t smem = 0;
    std::vector<void *> owned;
    const int *fit_k = nullptr;          // fitting tables (device)
    const T *fit_w = nullptr;
    unsigned char *multi_buf = nullptr;  // scratch of apply_multi (allocated on first use)
    size_t multi_stride = 0;

    size_t sm_fixed = 0;  // dynamic shared memory of every phase but the WFS tiles
    size_t sm_base = 0;   // of the layer and WFS phases alone (before the P^T bands)
    size_t sm_layer_ = 0; // of the layer phases alone
    std::vector<void *> band_owned;  // device tables of the P^T bands (replaced by plan_bands)
    int band_rows_large = 0, band_rows_small = 0;

    explicit Impl(const Plan &p) : P(p) {}

    // WFS tile bytes: per-layer halo values and the weighted slopes
    size_t wfs_bytes(int ty, int tx) const
    {
        return ((size_t)P.L * (ty + 2) * (tx + 2) + 2 * (size_t)(ty + 1) * (tx + 1)) * sizeof(T);
    }

    // WFS tiles of ty x tx pupil nodes on every sensor's grid: tiles per row
    // and the cumulative work-item count per sensor
    void set_tiles(Geo<T> &G, int ty, int tx) const
    {
        G.tile_y = ty;
        G.tile_x = tx;
        G.gs_tile0[0] = 0;
        for (int g = 0; g < P.G; g++) {
            G.gs_tiles_x[g] = (P.gm[g] + tx - 1) / tx;
            G.gs_tile0[g + 1] = G.gs_tile0[g] + G.gs_tiles_x[g] * ((P.gm[g] + ty - 1) / ty);
        }
    }

    // WFS tile shape: a square tile if the caller fixed one, else the shape
    // (8..32 nodes per side) whose work per round of `ctas` CTAs is least
    // among those whose shared memory fits
    int tiles_for(int ctas, int *ty_out, int *tx_out) const override
    {
        double best = 1e300;
        *ty_out = *tx_out = 0;
        const int cand[4] = {8, 16, 24, 32};
        for (int a = 0; a < 4; a++)
            for (int c = 0; c < 4; c++) {
                int ty = cand[a], tx = cand[c];
                if (P.geom.tile) ty = tx = P.geom.tile;
                if (wfs_bytes(ty, tx) > 200 * 1024) continue;
                int tiles = 0;
                for (int g = 0; g < P.G; g++) tiles += ((P.gm[g] + ty - 1) / ty) * ((P.gm[g] + tx - 1) / tx);
                const int rounds = (tiles + ctas - 1) / ctas;
                const double cost = rounds * ((double)(ty + 2) * (tx + 2) + 64.0);
                if (cost < best - 1e-9) {
                    best = cost;
                    *ty_out = ty;
                    *tx_out = tx;
                }
            }
        return *ty_out ? FEWHA_OK : FEWHA_ERR_GEOMETRY;
    }

    size_t smem_for(int ty, int tx) const override { return std::max(sm_fixed, wfs_bytes(ty, tx)); }
    size_t args_size() const override { return sizeof(Args<T, S>); }
    int precision_id() const override
    {
        return sizeof(T) == 8 ? FEWHA_F64 : (sizeof(S) == 2 ? FEWHA_BF16S : FEWHA_F32);
    }
    ~Impl() override
    {
        for (void *q : owned) cudaFree(q);
        for (void *q : band_owned) cudaFree(q);
    }

    template <typename U>
    int up(const std::vector<U> &v, const U **d)
    {
        U *dd;
        int st = upload(v, &dd);
        if (dd) owned.push_back(dd);
        *d = dd;
        return st;
    }
    template <typename U>
    int upb(const std::vector<U> &v, const U **d)  // a P^T band table (replaced by plan_bands)
    {
        U *dd;
        int st = upload(v, &dd);
        if (dd) band_owned.push_back(dd);
        *d = dd;
        return st;
    }
    template <typename U>
    int alloc(size_t count, U **d)
    {
        if (cudaMalloc(d, count * sizeof(U)) != cudaSuccess) return FEWHA_ERR_NOMEM;
        owned.push_back(*d);
        CK(cudaMemset(*d, 0, count * sizeof(U)));
        return FEWHA_OK;
    }

    // P^T work items and their tables: bands of rows_large layer rows on the
    // largest layers and rows_small on the smaller ones (at most kBandOutputs
    // outputs each); with the staging groups, tap lists and the shared memory
    // they need.  Replaces the tables of an earlier call.
    int plan_bands(int rows_large, int rows_small)
    {
        if (rows_large < 1 || rows_small < 1) return FEWHA_ERR_ARG;
        Geo<T> &G = base.geo;
        int st;
        int nmax = 0;
        for (int l = 0; l < P.L; l++) nmax = std::max(nmax, P.geom.layers[l].n);
        for (void *q : band_owned) cudaFree(q);
        band_owned.clear();
        // bands of BR rows with BR * n_l <= kBandOutputs outputs; by default 8
        // rows on the largest layers and 4 on the smaller ones (their coarser
        // grid touches about twice as many pupil rows per layer row, so a
        // half-height band balances the staged work)
        std::vector<int> bl, br0, brs;
        int n_largest = 0;
        for (int l = 0; l < P.L; l++) n_largest = std::max(n_largest, P.geom.layers[l].n);
        for (int l = 0; l < P.L; l++) {
            const int n = P.geom.layers[l].n;
            int BR = std::max(1, std::min(n, std::min(kBandOutputs / n, n < n_largest ? rows_small : rows_large)));
            for (int a0 = 0; a0 < n; a0 += BR) {
                bl.push_back(l);
                br0.push_back(a0);
                brs.push_back(std::min(BR, n - a0));
            }
        }
        G.nbands = (int)bl.size();
        std::vector<int> bilo((size_t)P.G * G.nbands), bihi((size_t)P.G * G.nbands);
        int max_rows = 1, max_rows_sum = 1;
        std::vector<int> rows_sum(G.nbands, 0);
        for (int g = 0; g < P.G; g++)
            for (int w = 0; w < G.nbands; w++) {
                int lo = P.gm[g], hi = 0;
                size_t by = ((size_t)g * P.L + bl[w]) * 2 + 1;
                for (int a = br0[w]; a < br0[w] + brs[w]; a++) {
                    int alo = P.alo[by * FEWHA_MAX_GRID + a], ahi = P.ahi[by * FEWHA_MAX_GRID + a];
                    if (alo < ahi) {
                        lo = std::min(lo, alo);
                        hi = std::max(hi, ahi);
                    }
                }
                if (lo >= hi) lo = hi = 0;
                bilo[(size_t)g * G.nbands + w] = lo;
                bihi[(size_t)g * G.nbands + w] = hi;
                max_rows = std::max(max_rows, hi - lo);
                rows_sum[w] += hi - lo;
                max_rows_sum = std::max(max_rows_sum, rows_sum[w]);
            }
        if ((st = upb(bl, &G.band_layer)) || (st = upb(br0, &G.band_row0)) || (st = upb(brs, &G.band_rows)) ||
            (st = upb(bilo, &G.band_ilo)) || (st = upb(bihi, &G.band_ihi)))
            return st;
        // band_gather stages rows_chunk psi rows and their x-contraction
        // (all guide stars of a band at once when they fit, else in groups)
        const size_t row_bytes = (size_t)(P.m_max + nmax) * sizeof(T);
        const size_t smem_cap = 200 * 1024;  // 227 KB per CTA minus the static shared memory
        size_t smem = sm_base;
        size_t want = (size_t)max_rows_sum * row_bytes;
        if (want > smem) smem = std::min(want, smem_cap);
        G.rows_chunk = (int)std::min<size_t>(max_rows_sum, smem / row_bytes);
        if (smem > smem_cap || G.rows_chunk < max_rows) return FEWHA_ERR_GEOMETRY;
        {
            // guide stars of each band in groups of consecutive guide stars whose
            // pupil rows fit rows_chunk staged rows
            std::vector<int> gend((size_t)P.G * G.nbands), gc((size_t)P.G * G.nbands), gr((size_t)P.G * G.nbands);
            for (int w = 0; w < G.nbands; w++)
                for (int g0 = 0, g1; g0 < P.G; g0 = g1) {
                    int rows_tot = 0;
                    for (g1 = g0; g1 < P.G; g1++) {
                        const size_t i = (size_t)g1 * G.nbands + w;
                        if (rows_tot + bihi[i] - bilo[i] > G.rows_chunk) break;
                        rows_tot += bihi[i] - bilo[i];
                    }
                    if (g1 == g0) return FEWHA_ERR_GEOMETRY;  // rows_chunk >= max_rows
                    for (int g = g0, c = 0, r = 0; g < g1; g++) {
                        const size_t i = (size_t)g * G.nbands + w;
                        gend[i] = g1;
                        gc[i] = c;
                        gr[i] = r;
                        c += (bihi[i] - bilo[i]) * P.gm[g];
                        r += bihi[i] - bilo[i];
                    }
                }
            if ((st = upb(gend, &G.band_gend)) || (st = upb(gc, &G.band_gc)) || (st = upb(gr, &G.band_gr))) return st;
            // y-contraction lists: for band row r of band w and the group that
            // starts at g0, the staged row (gr + pupil row - ilo) and weight of
            // each tap, guide star after guide star
            int ybr = 1, ymax = 1;
            for (int w = 0; w < G.nbands; w++) ybr = std::max(ybr, brs[w]);
            auto ytaps = [&](int w, int g, int r, std::vector<std::pair<int, double>> *out) {
                const size_t t = ((size_t)g * P.L + bl[w]) * 2 + 1;
                const int a = br0[w] + r, lo = P.alo[t * FEWHA_MAX_GRID + a], hi = P.ahi[t * FEWHA_MAX_GRID + a];
                const size_t i = (size_t)g * G.nbands + w;
                int cnt = 0;
                const size_t tb = P.tab(g, bl[w], 1);
                for (int j = lo; j < hi; j++, cnt++) {
                    if (!out) continue;
                    const double w0 = P.fw[tb + j];
                    out->push_back({gr[i] + (j - bilo[i]), P.fk[tb + j] == a ? 1.0 - w0 : w0});
                }
                return cnt;
            };
            for (int w = 0; w < G.nbands; w++)
                for (int g0 = 0; g0 < P.G; g0 = gend[(size_t)g0 * G.nbands + w])
                    for (int r = 0; r < brs[w]; r++) {
                        int c = 0;
                        for (int g = g0; g < gend[(size_t)g0 * G.nbands + w]; g++) c += ytaps(w, g, r, nullptr);
                        ymax = std::max(ymax, c);
                    }
            std::vector<int> ycnt((size_t)G.nbands * P.G * ybr, 0), yrow(ycnt.size() * ymax, 0);
            std::vector<T> yw(ycnt.size() * ymax, T(0));
            for (int w = 0; w < G.nbands; w++)
                for (int g0 = 0; g0 < P.G; g0 = gend[(size_t)g0 * G.nbands + w])
                    for (int r = 0; r < brs[w]; r++) {
                        std::vector<std::pair<int, double>> taps;
                        for (int g = g0; g < gend[(size_t)g0 * G.nbands + w]; g++) ytaps(w, g, r, &taps);
                        const size_t e = ((size_t)w * P.G + g0) * ybr + r;
                        ycnt[e] = (int)taps.size();
                        for (size_t t = 0; t < taps.size(); t++) {
                            yrow[e * ymax + t] = taps[t].first;
                            yw[e * ymax + t] = (T)taps[t].second;
                        }
                    }
            G.ybr = ybr;
            G.ymax = ymax;
            if ((st = upb(ycnt, &G.band_ycnt)) || (st = upb(yrow, &G.band_yrow)) || (st = upb(yw, &G.band_yw)))
                return st;
        }
        size_t sm_fixed = std::max(sm_layer_, std::min(want, smem_cap));
        // P^T x weight tables of one band (all guide stars) staged beside the
        // psi rows when kTabPT entries per thread and the shared memory suffice
        const size_t tab_entries = (size_t)P.G * nmax;
        const size_t tab_bytes = tab_entries * (kAdjW * sizeof(T) + 2 * sizeof(int));
        const size_t gather_bytes = (size_t)G.rows_chunk * row_bytes + tab_bytes;
        G.stage_tab = 0;
        if (tab_entries <= (size_t)kTabPT * kThreads && gather_bytes <= smem_cap) {
            G.stage_tab = 1;
            smem = std::max(smem, gather_bytes);
            sm_fixed = std::max(sm_fixed, gather_bytes);
        }
        this->smem = smem;
        this->sm_fixed = sm_fixed;
        base.smem_bytes = smem;
        band_rows_large = rows_large;
        band_rows_small = rows_small;
        return FEWHA_OK;
    }

    int init(int grid) override
    {
        Geo<T> &G = base.geo;
        G.G = P.G;
        G.L = P.L;
        G.ns = P.ns;
        G.m = P.m;
        G.n = P.n;
        for (int g = 0; g < P.G; g++) {
            G.gs_ns[g] = P.gns[g];
            G.gs_m[g] = P.gm[g];
            G.gs_tab[g] = P.tab_off[g];
            G.gs_psi[g] = P.psi_off[g];
            G.gs_sl[g] = P.slope_off[g];
            G.gs_mask[g] = P.mask_off[g];
        }
        G.m_max = P.m_max;
        for (int l = 0; l < P.L; l++) {
            G.lay_n[l] = P.geom.layers[l].n;
            G.lay_J[l] = P.geom.layers[l].J;
            G.lay_off[l] = P.lay_off[l];
            G.inv_delta[l] = (T)(1.0 / P.geom.layers[l].delta);
        }
        G.lay_off[P.L] = P.lay_off[P.L];
        G.ll_off[0] = 0;
        for (int l = 0; l < P.L; l++) {
            const long h = P.geom.layers[l].n / 2;
            G.ll_off[l + 1] = G.ll_off[l] + h * h;
        }
        G.n_taps = (int)P.taps.size();
        for (int t = 0; t < kMaxT; t++) {
            G.h[t] = t < G.n_taps ? (T)P.taps[t] : T(0);
            G.g[t] = t < G.n_taps ? (T)(((t & 1) ? -1.0 : 1.0) * P.taps[G.n_taps - 1 - t]) : T(0);
        }
        // WFS tiles for the whole grid
        {
            int dev0, nsm0;
            CK(cudaGetDevice(&dev0));
            CK(cudaDeviceGetAttribute(&nsm0, cudaDevAttrMultiProcessorCount, dev0));
            int ty, tx;
            if (tiles_for(grid > 0 ? grid : nsm0, &ty, &tx)) return FEWHA_ERR_GEOMETRY;
            set_tiles(G, ty, tx);
        }
        int st;
        if ((st = up(P.fk, &G.fk)) || (st = up(P.alo, &G.alo)) || (st = up(P.ahi, &G.ahi))) return st;
        std::vector<T> fw(P.fw.begin(), P.fw.end());
        std::vector<T> ad(P.alpha_d.begin(), P.alpha_d.end());
        std::vector<T> one(P.n, T(1));
        if ((st = up(fw, &G.fw)) || (st = up(weight_table(), &G.wmask)) || (st = up(ad, &G.alpha_d)) ||
            (st = up(one, &G.invJ)))
            return st;
        for (int l = 0; l < P.L; l++) {
            int lg = 0;
            while ((1 << lg) < P.geom.layers[l].n) lg++;
            G.lay_lg[l] = lg;
        }
        // compact P_g^T weights: per layer node, its pupil-node range and weights
        {
            size_t nt = (size_t)P.G * P.L * 2 * FEWHA_MAX_GRID;
            std::vector<int> alo(nt, 0), acnt(nt, 0);
            std::vector<T> aw(nt * kAdjW, T(0));
            for (size_t t = 0; t < (size_t)P.G * P.L * 2; t++)
                for (int k = 0; k < FEWHA_MAX_GRID; k++) {
                    int lo = P.alo[t * FEWHA_MAX_GRID + k], hi = P.ahi[t * FEWHA_MAX_GRID + k];
                    if (hi - lo > kAdjW) return FEWHA_ERR_GEOMETRY;
                    alo[t * FEWHA_MAX_GRID + k] = lo;
                    acnt[t * FEWHA_MAX_GRID + k] = hi - lo;
                    const size_t tb = P.tab((int)(t / (2 * P.L)), (int)((t / 2) % P.L), (int)(t % 2));
                    for (int j = lo; j < hi; j++) {
                        double w0 = P.fw[tb + j];
                        aw[(t * FEWHA_MAX_GRID + k) * kAdjW + (j - lo)] = (T)(P.fk[tb + j] == k ? 1.0 - w0 : w0);
                    }
                }
            if ((st = up(alo, &G.adj_lo)) || (st = up(acnt, &G.adj_cnt)) || (st = up(aw, &G.adj_w))) return st;
            {
                std::vector<T> fw2(P.fit_w.begin(), P.fit_w.end());
                if ((st = up(P.fit_k, &fit_k)) || (st = up(fw2, &fit_w))) return st;
            }
        }
        if ((st = alloc((size_t)P.n, &base.nodal)) || (st = alloc((size_t)P.n, &base.u)) ||
            (st = alloc((size_t)P.n, &base.wq)) ||
            (st = alloc((size_t)P.psi_off[P.G], &base.psi)) || (st = alloc((size_t)P.n / 4 + 1, &base.ll)) ||
            (st = alloc((size_t)kSlots * kMaxCtas, &base.part)) || (st = alloc((size_t)1, &base.rec)))
            return st;
        if constexpr (std::is_same<T, S>::value) {
            base.nodal_t = base.nodal;
            base.psi_t = base.psi;
        } else {  // BF16 storage: the residual replacement stores its intermediates in T
            if ((st = alloc((size_t)P.n, &base.nodal_t)) || (st = alloc((size_t)P.psi_off[P.G], &base.psi_t)))
                return st;
        }
        // launch geometry: dynamic shared memory = max over phases
        int nmax = 0;
        for (int l = 0; l < P.L; l++) nmax = std::max(nmax, P.geom.layers[l].n);
        size_t sm_layer = (size_t)nmax * (nmax + 1) * sizeof(T);  // pitch n + 1
        G.pingpong = sizeof(T) == 4 ? 1 : 0;  // FP32: second buffer for out-of-place DWT passes
        if (G.pingpong) sm_layer *= 2;
        const size_t sm_wfs = wfs_bytes(G.tile_y, G.tile_x);
        // tiles of the finest wavelet level (analysis: input window and row-pass
        // output; synthesis: four subband windows and the column-pass output)
        size_t sm_fine = 0;
        {
            const int Lt = (int)P.taps.size();
            for (int l = 0; l < P.L; l++) {
                const size_t t = std::min(kFineTile, P.geom.layers[l].n / 2);
                const size_t ia = (2 * t + Lt - 2), wa = t + Lt / 2 - 1;
                sm_fine = std::max(sm_fine, std::max(ia * ia + ia * 2 * t, 4 * wa * wa + 2 * t * 2 * wa) * sizeof(T));
            }
        }
        sm_layer = std::max(sm_layer, sm_fine);
        smem = std::max(sm_layer, sm_wfs);
        sm_base = smem;
        sm_layer_ = sm_layer;
        if ((st = plan_bands(8, 4))) return st;
        int dev, nsm;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        // the attribute allows the cap, so that plan_bands may change smem later
        auto setattr = [&](const void *f) {
            return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        };
        CK(setattr((const void *)k_apply_idwt<T, S>));
        CK(setattr((const void *)k_wfs<T, S, false>));
        CK(setattr((const void *)k_wfs<T, S, true>));
        CK(setattr((const void *)k_gather<T, S>));
        CK(setattr((const void *)k_fdwt<T, S, false>));
        CK(setattr((const void *)k_fdwt<T, S, true>));
        CK(setattr((const void *)k_rhs_wfs<T, S>));
        CK(setattr((const void *)k_rhs_D1<T, S>));
        CK(setattr((const void *)k_rhs_update<T, S>));
        CK(setattr((const void *)k_rhs_gather<T, S>));
        CK(setattr((const void *)k_init<T, S>));
        CK(setattr((const void *)k_UA1<T, S>));
        CK(setattr((const void *)k_A2<T, S>));
        CK(setattr((const void *)k_B<T, S>));
        CK(setattr((const void *)k_C<T, S>));
        CK(setattr((const void *)k_D1<T, S>));
        CK(setattr((const void *)k_D2E<T, S>));
        CK(setattr((const void *)k_finish<T, S>));
        CK(setattr((const void *)k_TU<T, S>));
        CK(setattr((const void *)k_TA2<T, S>));
        CK(setattr((const void *)k_TB<T, S>));
        CK(setattr((const void *)k_TC<T, S>));
        CK(setattr((const void *)k_TD1<T, S>));
        CK(setattr((const void *)k_TE<T, S>));
        CK(setattr((const void *)k_solve_persistent<T, S, false>));
        CK(setattr((const void *)k_solve_persistent<T, S, true>));
        CK(setattr((const void *)k_solve_persistent<T, S, false, true>));
        CK(setattr((const void *)k_solve_persistent<T, S, true, true>));
        CK(cudaFuncSetAttribute((const void *)k_solve_batched<T, S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024));
        CK(cudaFuncSetAttribute((const void *)k_solve_batched<T, S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024));
        for (const void *f : {(const void *)k_multi_idwt<T, S>, (const void *)k_multi_wfs<T, S>,
                              (const void *)k_multi_gather<T, S>, (const void *)k_multi_fdwt<T, S>})
            CK(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        int per_sm = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_persistent<T, S, false>, kThreads, smem));
        if (per_sm < 1) return FEWHA_ERR_CUDA;
        {
            int per_sm_tr = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_tr, k_solve_persistent<T, S, true>, kThreads,
                                                             smem));
            per_sm = std::min(per_sm, per_sm_tr);
            if (per_sm < 1) return FEWHA_ERR_CUDA;
        }
        ncta = grid > 0 ? grid : nsm;
        if (ncta > nsm * per_sm) ncta = nsm * per_sm;
        if (ncta > kMaxCtas) ncta = kMaxCtas;
        base.timeout_ns = 1000000000ull;
        base.ncta = ncta;
        base.cta0 = 0;
        base.smem_bytes = smem;
        return FEWHA_OK;
    }

    int set_bands(int rows_large, int rows_small) override
    {
        if (rows_large < 1 || rows_small < 1) return FEWHA_ERR_ARG;
        CK(cudaDeviceSynchronize());  // the tables may be in use
        const int ol = band_rows_large, os = band_rows_small;
        int st = plan_bands(rows_large, rows_small);
        if (st != FEWHA_OK) {
            plan_bands(ol, os);  // keep the earlier plan
            return st;
        }
        return FEWHA_OK;
    }

    void launch_info(fewha_launch_info *out) const override
    {
        out->ctas = ncta;
        out->threads = kThreads;
        out->smem_bytes = (long)smem;
        out->split_levels = ncta >= 2 * P.L ? 1 : 0;
        out->staged_tables = base.geo.stage_tab;
        out->wfs_tile_y = base.geo.tile_y;
        out->wfs_tile_x = base.geo.tile_x;
        out->pt_bands = base.geo.nbands;
        out->pt_rows_chunk = base.geo.rows_chunk;
        out->pt_rows_large = band_rows_large;
        out->pt_rows_small = band_rows_small;
    }

    int get_invJ(double *host) const override
    {
        std::vector<T> v(P.n);
        CK(cudaMemcpy(v.data(), base.geo.invJ, P.n * sizeof(T), cudaMemcpyDeviceToHost));
        for (long i = 0; i < P.n; i++) host[i] = (double)v[i];
        return FEWHA_OK;
    }

    // C_eta^{-1} per slope: 1/sigma_g^2 on lit subapertures, 0 elsewhere
    std::vector<T> weight_table() const
    {
        std::vector<T> wm((size_t)P.mask_off[P.G]);
        for (int g = 0; g < P.G; g++)
            for (long i = P.mask_off[g]; i < P.mask_off[g + 1]; i++)
                wm[i] = P.mask[i] ? (T)P.geom.gs[g].weight : T(0);
        return wm;
    }

    int set_weights() override
    {
        const std::vector<T> wm = weight_table();
        CK(cudaMemcpy(const_cast<T *>(base.geo.wmask), wm.data(), wm.size() * sizeof(T), cudaMemcpyHostToDevice));
        return FEWHA_OK;
    }

    int set_invJ(const std::vector<double> &invJ) override
    {
        std::vector<T> v(invJ.begin(), invJ.end());
        CK(cudaMemcpy(const_cast<T *>(base.geo.invJ), v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
        return FEWHA_OK;
    }

    void set_timeout(unsigned long long ns) override { base.timeout_ns = ns; }

    void set_trace(unsigned long long *buf, int cap) override
    {
        base.trace = buf;
        base.trace_cap = buf ? cap : 0;
    }

    int launch_check() { return cudaGetLastError() == cudaSuccess ? FEWHA_OK : FEWHA_ERR_CUDA; }

    int apply(const void *x, void *y, cudaStream_t s) override
    {
        Args<T, S> A = base;
        A.x = static_cast<const T *>(x);
        A.y = static_cast<T *>(y);
        CK(cudaMemsetAsync(A.rec, 0, offsetof(Record, rz), s));
        k_apply_idwt<T, S><<<ncta, kThreads, smem, s>>>(A);
        k_wfs<T, S, false><<<ncta, kThreads, smem, s>>>(A);
        k_gather<T, S><<<ncta, kThreads, smem, s>>>(A);
        k_fdwt<T, S, false><<<ncta, kThreads, smem, s>>>(A);
        return launch_check();
    }

    int fit(const void *c, void *a, cudaStream_t s) override
    {
        if (!P.fit_ok) return FEWHA_ERR_GEOMETRY;
        Args<T, S> A = base;
        A.x = static_cast<const T *>(c);
        CK(cudaMemsetAsync(A.rec, 0, offsetof(Record, rz), s));
        k_apply_idwt<T, S><<<ncta, kThreads, smem, s>>>(A);  // nodal = W^{-1} c
        FitTab<T> F{};
        for (int l = 0; l < P.L; l++) {
            F.off[l] = P.lay_off[l];
            F.n[l] = P.geom.layers[l].n;
        }
        F.L = P.L;
        F.m = P.m;
        F.fk = fit_k;
        F.fw = fit_w;
        k_fit<T, S><<<(P.m * P.m + 255) / 256, 256, 0, s>>>(F, base.nodal, static_cast<T *>(a));
        return launch_check();
    }

    // MCAO fitting plan: device tables and work vectors of one mirror system
    struct McaoPlan {
        McaoArgs<T, S> M{};
        std::vector<void *> owned;
        ~McaoPlan()
        {
            for (void *q : owned) cudaFree(q);
        }
    };

    int mcao_create(const fewha_mcao_desc *d, void **out, long *n_act) override
    {
        if (d->n_dm < 1 || d->n_dm > FEWHA_MAX_DM || d->n_dir < 1 || d->n_dir > FEWHA_MAX_DIR)
            return FEWHA_ERR_ARG;
        const int m = P.m, L = P.L, D = d->n_dm, T_ = d->n_dir;
        int nmax = 0;
        for (int k = 0; k < D; k++) {
            if (d->dm_n[k] < 2 || !(d->dm_pitch[k] > 0) || !std::isfinite(d->dm_pitch[k]) ||
                !std::isfinite(d->dm_h[k]) || d->dm_h[k] < 0)
                return FEWHA_ERR_ARG;
            nmax = std::max(nmax, d->dm_n[k]);
        }
        for (int t = 0; t < T_; t++)
            if (!std::isfinite(d->dir_x[t]) || !std::isfinite(d->dir_y[t])) return FEWHA_ERR_ARG;
        // bilinear tables: pupil node j at x = -D/2 + j ds; layer node k at
        // (k - n/2) d_l; actuator i at (i - (n-1)/2) pitch
        std::vector<int> lk((size_t)T_ * L * 2 * m), dk((size_t)T_ * D * 2 * m);
        std::vector<T> lw(lk.size()), dw(dk.size());
        std::vector<int> alo((size_t)T_ * D * 2 * nmax, 0), ahi(alo.size(), 0);
        auto table = [&](double shift, double spacing, double centre, int n, int *k_out, T *w_out) {
            for (int j = 0; j < m; j++) {
                const double f = (-0.5 * P.geom.D + j * P.ds + shift) / spacing + centre;
                const int k = (int)std::floor(f);
                if (k < 0 || k + 1 > n - 1) return false;
                k_out[j] = k;
                w_out[j] = (T)(f - k);
            }
            return true;
        };
        for (int t = 0; t < T_; t++) {
            for (int l = 0; l < L; l++) {
                const fewha_layer &ly = P.geom.layers[l];
                for (int ax = 0; ax < 2; ax++) {
                    const size_t b = (((size_t)t * L + l) * 2 + ax) * m;
                    const double th = ax == 0 ? d->dir_x[t] : d->dir_y[t];
                    if (!table(th * ly.h, P.lay_d[l], 0.5 * ly.n, ly.n, &lk[b], &lw[b])) return FEWHA_ERR_GEOMETRY;
                }
            }
            for (int k = 0; k < D; k++)
                for (int ax = 0; ax < 2; ax++) {
                    const size_t b = (((size_t)t * D + k) * 2 + ax) * m;
                    const double th = ax == 0 ? d->dir_x[t] : d->dir_y[t];
                    if (!table(th * d->dm_h[k], d->dm_pitch[k], 0.5 * (d->dm_n[k] - 1), d->dm_n[k], &dk[b], &dw[b]))
                        return FEWHA_ERR_GEOMETRY;
                    const size_t rb = (((size_t)t * D + k) * 2 + ax) * nmax;
                    for (int i = 0; i < d->dm_n[k]; i++) {
                        int lo = m, hi = 0;
                        for (int j = 0; j < m; j++)
                            if (dk[b + j] == i || dk[b + j] + 1 == i) {
                                lo = std::min(lo, j);
                                hi = std::max(hi, j + 1);
                            }
                        if (lo >= hi) lo = hi = 0;
                        alo[rb + i] = lo;
                        ahi[rb + i] = hi;
                    }
                }
        }
        auto *pl = new McaoPlan();
        McaoArgs<T, S> &M = pl->M;
        M.L = L;
        M.D = D;
        M.ndir = T_;
        M.m = m;
        M.nmax = nmax;
        for (int l = 0; l < L; l++) {
            M.lay_off[l] = P.lay_off[l];
            M.lay_n[l] = P.geom.layers[l].n;
        }
        M.dm_off[0] = 0;
        for (int k = 0; k < D; k++) {
            M.dm_n[k] = d->dm_n[k];
            M.dm_off[k + 1] = M.dm_off[k] + (long)d->dm_n[k] * d->dm_n[k];
        }
        const long na = M.dm_off[D];
        int st = FEWHA_OK;
        auto put_i = [&](const std::vector<int> &v, const int **dst) {
            int *dd = nullptr;
            if (upload(v, &dd)) return false;
            pl->owned.push_back(dd);
            *dst = dd;
            return true;
        };
        auto put_t = [&](const std::vector<T> &v, const T **dst) {
            T *dd = nullptr;
            if (upload(v, &dd)) return false;
            pl->owned.push_back(dd);
            *dst = dd;
            return true;
        };
        auto make = [&](size_t bytes, void **dst) {
            if (cudaMalloc(dst, bytes) != cudaSuccess) return false;
            pl->owned.push_back(*dst);
            return true;
        };
        const int *c_lk, *c_dk, *c_alo, *c_ahi;
        const T *c_lw, *c_dw;
        void *r, *p, *q, *y, *part, *rec;
        if (!put_i(lk, &c_lk) || !put_t(lw, &c_lw) || !put_i(dk, &c_dk) || !put_t(dw, &c_dw) ||
            !put_i(alo, &c_alo) || !put_i(ahi, &c_ahi) || !make(na * sizeof(T), &r) || !make(na * sizeof(T), &p) ||
            !make(na * sizeof(T), &q) || !make((size_t)T_ * m * m * sizeof(T), &y) ||
            !make(2 * kMaxCtas * sizeof(double), &part) || !make(sizeof(Record), &rec))
            st = FEWHA_ERR_CUDA;
        if (st) {
            delete pl;
            return st;
        }
        M.lk = c_lk;
        M.lw = c_lw;
        M.dk = c_dk;
        M.dw = c_dw;
        M.alo = c_alo;
        M.ahi = c_ahi;
        M.r = static_cast<T *>(r);
        M.p = static_cast<T *>(p);
        M.q = static_cast<T *>(q);
        M.y = static_cast<T *>(y);
        M.part = static_cast<double *>(part);
        M.rec = static_cast<Record *>(rec);
        *out = pl;
        *n_act = na;
        return FEWHA_OK;
    }

    int mcao_fit(void *plan, const void *c, void *a, int iters, cudaStream_t s) override
    {
        if (iters < 0 || iters > FEWHA_MAX_ITER) return FEWHA_ERR_ARG;
        auto *pl = static_cast<McaoPlan *>(plan);
        Args<T, S> A = base;
        A.x = static_cast<const T *>(c);
        CK(cudaMemsetAsync(A.rec, 0, offsetof(Record, rz), s));
        k_apply_idwt<T, S><<<ncta, kThreads, smem, s>>>(A);  // nodal = W^{-1} c
        McaoArgs<T, S> M = pl->M;
        M.nodal = base.nodal;
        M.a = static_cast<T *>(a);
        M.iters = iters;
        M.timeout_ns = base.timeout_ns;
        CK(cudaMemsetAsync(M.rec, 0, sizeof(Record), s));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(ncta);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        CK(cudaLaunchKernelEx(&cfg, k_mcao_fit<T, S>, M));
        return launch_check();
    }

    void mcao_destroy(void *plan) override { delete static_cast<McaoPlan *>(plan); }

    int pol_slopes(const void *s_in, const void *a, void *s_out, cudaStream_t s) override
    {
        for (int g = 0; g < P.G; g++)  // the mirror's actuators sit on the geometry's pupil grid
            if (P.gns[g] != P.ns) return FEWHA_ERR_GEOMETRY;
        k_pol<T, S><<<256, 256, 0, s>>>(static_cast<const S *>(s_in), static_cast<const T *>(a),
                                        static_cast<S *>(s_out), P.G, P.ns);
        return launch_check();
    }

    int control(int closed, double gain, const void *am1, const void *ai, const void *af, void *an,
                cudaStream_t s) override
    {
        const int na = P.m * P.m;
        k_control<T><<<(na + 255) / 256, 256, 0, s>>>(closed, (T)gain, static_cast<const T *>(am1),
                                                      static_cast<const T *>(ai), static_cast<const T *>(af),
                                                      static_cast<T *>(an), na);
        return launch_check();
    }

    int apply_multi(const void *x, long ldx, void *y, long ldy, int nvec, cudaStream_t s) override
    {
        static_assert(sizeof(MultiArgs<T, S>) <= 32000, "kernel parameter size");
        if (nvec < 1 || nvec > kMaxVec || ldx < P.n || ldy < P.n) return FEWHA_ERR_ARG;
        auto up256 = [](size_t v) { return (v + 255) & ~(size_t)255; };
        if (!multi_buf) {
            multi_stride = up256((size_t)P.n * sizeof(S)) + up256((size_t)P.psi_off[P.G] * sizeof(S)) +
                           up256((size_t)P.n * sizeof(T));
            if (alloc(multi_stride * kMaxVec, &multi_buf)) return FEWHA_ERR_NOMEM;
        }
        const int per = std::max(1, ncta / nvec);
        int ty, tx;
        if (tiles_for(per, &ty, &tx)) return FEWHA_ERR_GEOMETRY;
        const size_t sm = smem_for(ty, tx);
        MultiArgs<T, S> M{};
        M.per = per;
        for (int v = 0; v < nvec; v++) {
            Args<T, S> A = base;
            unsigned char *b = multi_buf + (size_t)v * multi_stride;
            A.nodal = reinterpret_cast<S *>(b);
            A.psi = reinterpret_cast<S *>(b + up256((size_t)P.n * sizeof(S)));
            A.u = reinterpret_cast<T *>(b + up256((size_t)P.n * sizeof(S)) + up256((size_t)P.psi_off[P.G] * sizeof(S)));
            A.part = base.part + (size_t)v * per;  // disjoint partial-sum columns
            A.x = static_cast<const T *>(x) + (size_t)v * ldx;
            A.y = static_cast<T *>(y) + (size_t)v * ldy;
            A.cta0 = v * per;
            A.ncta = per;
            set_tiles(A.geo, ty, tx);
            A.smem_bytes = sm;
            A.trace = nullptr;
            A.trace_cap = 0;
            M.a[v] = A;
        }
        CK(cudaMemsetAsync(base.rec, 0, offsetof(Record, rz), s));
        const int grid = per * nvec;
        k_multi_idwt<T, S><<<grid, kThreads, sm, s>>>(M);
        k_multi_wfs<T, S><<<grid, kThreads, sm, s>>>(M);
        k_multi_gather<T, S><<<grid, kThreads, sm, s>>>(M);
        k_multi_fdwt<T, S><<<grid, kThreads, sm, s>>>(M);
        return launch_check();
    }

    int apply_in_scratch(const void *x, void *y, void *scratch, size_t bytes, cudaStream_t s) override
    {
        // layout: record | partial sums | nodal layers | adjoint wavefronts | P^T output
        auto up256 = [](size_t v) { return (v + 255) & ~(size_t)255; };
        const size_t o_rec = 0;
        const size_t o_part = up256(o_rec + sizeof(Record));
        const size_t o_nodal = up256(o_part + (size_t)kSlots * kMaxCtas * sizeof(double));
        const size_t o_psi = up256(o_nodal + (size_t)P.n * sizeof(S));
        const size_t o_u = up256(o_psi + (size_t)P.psi_off[P.G] * sizeof(S));
        const size_t need = up256(o_u + (size_t)P.n * sizeof(T));
        if (need > bytes) return FEWHA_ERR_SCRATCH;
        unsigned char *base_p = static_cast<unsigned char *>(scratch);
        Args<T, S> A = base;
        A.rec = reinterpret_cast<Record *>(base_p + o_rec);
        A.part = reinterpret_cast<double *>(base_p + o_part);
        A.nodal = reinterpret_cast<S *>(base_p + o_nodal);
        A.psi = reinterpret_cast<S *>(base_p + o_psi);
        A.u = reinterpret_cast<T *>(base_p + o_u);
        A.trace = nullptr;
        A.trace_cap = 0;
        A.x = static_cast<const T *>(x);
        A.y = static_cast<T *>(y);
        // the record's flags must start at zero; the other buffers are fully
        // overwritten before they are read
        CK(cudaMemsetAsync(A.rec, 0, offsetof(Record, rz), s));
        k_apply_idwt<T, S><<<ncta, kThreads, smem, s>>>(A);
        k_wfs<T, S, false><<<ncta, kThreads, smem, s>>>(A);
        k_gather<T, S><<<ncta, kThreads, smem, s>>>(A);
        k_fdwt<T, S, false><<<ncta, kThreads, smem, s>>>(A);
        return launch_check();
    }

    int rhs(const void *sl, void *b, cudaStream_t s) override
    {
        Args<T, S> A = base;
        A.slopes = static_cast<const S *>(sl);
        A.y = static_cast<T *>(b);
        CK(cudaMemsetAsync(A.rec, 0, offsetof(Record, rz), s));
        k_wfs<T, S, true><<<ncta, kThreads, smem, s>>>(A);
        k_gather<T, S><<<ncta, kThreads, smem, s>>>(A);
        k_fdwt<T, S, true><<<ncta, kThreads, smem, s>>>(A);
        return launch_check();
    }

    Args<T, S> solve_args(const void *sl, void *c, const fewha_state *st, const fewha_solve_opts *o,
                          fewha_stats *stats) const
    {
        Args<T, S> A = base;
        A.slopes = static_cast<const S *>(sl);
        A.c = static_cast<T *>(c);
        A.r = static_cast<T *>(st->r_prev);
        A.b_prev = static_cast<T *>(st->b_prev);
        A.P = static_cast<T *>(st->basis_P);
        A.Q = static_cast<T *>(st->basis_Q);
        A.pq = st->basis_pq;
        A.meta = st->meta;
        A.kcap = st->k_cap;
        A.max_iter = o->max_iter;
        A.rtol = o->rtol;
        A.augmented = o->augmented ? 1 : 0;
        A.recycle_all = o->recycle_mode == FEWHA_RECYCLE_ALL ? 1 : 0;
        A.true_res_every = o->true_res_every;
        A.rhs_in_state = o->rhs_in_state ? 1 : 0;
        A.c_out = static_cast<T *>(o->c_out);
        A.stats = stats;
        return A;
    }

    int batch_args(void *out, const void *sl, void *c, const fewha_state *st, const fewha_solve_opts *o,
                   fewha_stats *stats, int cta0, int nct, int ty, int tx, size_t sm) const override
    {
        Args<T, S> A = solve_args(sl, c, st, o, stats);
        A.c_out = nullptr;  // the batch calls have no second destination
        A.cta0 = cta0;
        A.ncta = nct;
        set_tiles(A.geo, ty, tx);
        A.smem_bytes = sm;
        A.trace = nullptr;
        A.trace_cap = 0;
        std::memcpy(out, &A, sizeof(A));
        return FEWHA_OK;
    }

    int batch_capacity(size_t sm, int *max_ctas) const override
    {
        int dev, nsm, per_sm = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        int per_sm_tr = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_batched<T, S, false>, kThreads, sm));
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_tr, k_solve_batched<T, S, true>, kThreads, sm));
        *max_ctas = std::min(nsm * std::min(per_sm, per_sm_tr), kMaxCtas);
        return FEWHA_OK;
    }

    int launch_batched(const void *d_args, const int *d_map, int n, int total, size_t sm, int nrounds,
                       Record *brec, int true_res, cudaStream_t s) const override
    {
        const Args<T, S> *args = static_cast<const Args<T, S> *>(d_args);
        k_batch_reset<T, S><<<(n + 255) / 256, 256, 0, s>>>(args, n, brec);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(total);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        // a round may run as long as one time step of its slowest instance
        const unsigned long long to = base.timeout_ns * 4;
        if (true_res)
            CK(cudaLaunchKernelEx(&cfg, k_solve_batched<T, S, true>, args, d_map, nrounds, total, brec, to));
        else
            CK(cudaLaunchKernelEx(&cfg, k_solve_batched<T, S, false>, args, d_map, nrounds, total, brec, to));
        return cudaGetLastError() == cudaSuccess ? FEWHA_OK : FEWHA_ERR_CUDA;
    }

    int solve(const void *sl, void *c, const fewha_state *st, const fewha_solve_opts *o,
              fewha_stats *stats, cudaStream_t s) override
    {
        Args<T, S> A = solve_args(sl, c, st, o, stats);
        CK(cudaMemsetAsync(A.rec, 0, offsetof(Record, rz), s));
        CK(cudaMemsetAsync(&A.rec->bar, 0, sizeof(Bar), s));
        if (A.trace) CK(cudaMemsetAsync(A.trace, 0, (size_t)A.trace_cap * 4 * sizeof(unsigned long long), s));
        if (o->launch_mode == FEWHA_LAUNCH_PERSISTENT) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(ncta);
            cfg.blockDim = dim3(kThreads);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            const bool tr = A.true_res_every > 0, ris = A.rhs_in_state != 0;
            if (tr && ris)
                CK(cudaLaunchKernelEx(&cfg, k_solve_persistent<T, S, true, true>, A));
            else if (tr)
                CK(cudaLaunchKernelEx(&cfg, k_solve_persistent<T, S, true>, A));
            else if (ris)
                CK(cudaLaunchKernelEx(&cfg, k_solve_persistent<T, S, false, true>, A));
            else
                CK(cudaLaunchKernelEx(&cfg, k_solve_persistent<T, S, false>, A));
            return launch_check();
        }
        k_rhs_wfs<T, S><<<ncta, kThreads, smem, s>>>(A);
        k_rhs_gather<T, S><<<ncta, kThreads, smem, s>>>(A);
        k_rhs_D1<T, S><<<ncta, kThreads, smem, s>>>(A);
        k_rhs_update<T, S><<<ncta, kThreads, smem, s>>>(A);
        k_init<T, S><<<ncta, kThreads, smem, s>>>(A);
        for (int k = 0; k < A.max_iter; k++) {
            k_UA1<T, S><<<ncta, kThreads, smem, s>>>(A, k);
            k_A2<T, S><<<ncta, kThreads, smem, s>>>(A, k);
            k_B<T, S><<<ncta, kThreads, smem, s>>>(A, k);
            k_C<T, S><<<ncta, kThreads, smem, s>>>(A, k);
            k_D1<T, S><<<ncta, kThreads, smem, s>>>(A, k);
            k_D2E<T, S><<<ncta, kThreads, smem, s>>>(A, k);
            if (A.true_res_every > 0 && (k + 1) % A.true_res_every == 0) {
                k_TU<T, S><<<ncta, kThreads, smem, s>>>(A);
                k_TA2<T, S><<<ncta, kThreads, smem, s>>>(A);
                k_TB<T, S><<<ncta, kThreads, smem, s>>>(A);
                k_TC<T, S><<<ncta, kThreads, smem, s>>>(A);
                k_TD1<T, S><<<ncta, kThreads, smem, s>>>(A);
                k_TE<T, S><<<ncta, kThreads, smem, s>>>(A, k);
            }
        }
        k_finish<T, S><<<1, kThreads, smem, s>>>(A);
        return launch_check();
    }
};


ImplBase *make_impl_f64(const Plan &p);
// Working-precision implementation of a handle and the device it was created
// on (defined with the C ABI).
ImplBase *handle_impl(void *handle);
int handle_device(const void *handle);
// Device address of the allocation-free entry point's static scratch on the
// current device; the first call on a device loads the module that holds it.
int noalloc_prepare();
ImplBase *make_impl_f32(const Plan &p);
ImplBase *make_impl_bf16(const Plan &p);

}  // namespace fewha
