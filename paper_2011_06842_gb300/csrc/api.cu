// libfewha: the C ABI (include/fewha.h) of the GB300 augmented FEWHA hot
// path.  The handle plans the geometry on the host, owns constant tables and
// scratch on the current device, and launches the kernels of one precision.
#include <cuda_runtime.h>

#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "kernels.cuh"

namespace fewha {

struct Handle {
    Plan plan;
    int device = 0;
    std::unique_ptr<ImplBase> f64;              // always present (setup of J)
    std::unique_ptr<ImplBase> work;             // working precision (== f64 for FEWHA_F64)
    ImplBase *w() { return work ? work.get() : f64.get(); }
};

ImplBase *handle_impl(void *handle) { return handle ? static_cast<Handle *>(handle)->w() : nullptr; }

// Modified Jacobi preconditioner (Sec. 4): J = alpha D + t_band, with t_band
// the mean over sampled coefficients of the data term's diagonal
// e_i^T M e_i - alpha D_ii, computed with the FP64 operator.
static int build_precond(Handle &h, std::vector<double> &invJ)
{
    const Plan &P = h.plan;
    double *x = nullptr, *y = nullptr;
    if (cudaMalloc(&x, P.n * sizeof(double)) != cudaSuccess) return FEWHA_ERR_NOMEM;
    if (cudaMalloc(&y, P.n * sizeof(double)) != cudaSuccess) {
        cudaFree(x);
        return FEWHA_ERR_NOMEM;
    }
    std::vector<double> sum(P.n_classes, 0.0);
    std::vector<int> cnt(P.n_classes, 0);
    int st = FEWHA_OK;
    const double one = 1.0;
    for (size_t s = 0; s < P.sample_idx.size() && st == FEWHA_OK; s++) {
        long i = P.sample_idx[s];
        if (cudaMemset(x, 0, P.n * sizeof(double)) != cudaSuccess ||
            cudaMemcpy(x + i, &one, sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            st = FEWHA_ERR_CUDA;
            break;
        }
        st = h.f64->apply(x, y, 0);
        double yi = 0;
        if (st == FEWHA_OK && cudaMemcpy(&yi, y + i, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = FEWHA_ERR_CUDA;
        sum[P.sample_class[s]] += yi - P.alpha_d[i];
        cnt[P.sample_class[s]] += 1;
    }
    cudaFree(x);
    cudaFree(y);
    if (st) return st;
    invJ.resize(P.n);
    for (long i = 0; i < P.n; i++) {
        int c = P.coef_class[i];
        double t = cnt[c] ? sum[c] / cnt[c] : 0.0;
        double J = P.alpha_d[i] + t;
        if (!(J > 0)) return FEWHA_ERR_GEOMETRY;
        invJ[i] = 1.0 / J;
    }
    return FEWHA_OK;
}

}  // namespace fewha

using namespace fewha;

extern "C" {

int fewha_create(const fewha_geometry *geom, void **out)
{
    if (!geom || !out) return FEWHA_ERR_ARG;
    *out = nullptr;
    Handle *h = new (std::nothrow) Handle();
    if (!h) return FEWHA_ERR_NOMEM;
    int st = build_plan(*geom, h->plan);
    if (st == FEWHA_OK && cudaGetDevice(&h->device) != cudaSuccess) st = FEWHA_ERR_CUDA;
    if (st == FEWHA_OK) {
        h->f64.reset(make_impl_f64(h->plan));
        st = h->f64->init(geom->grid);
    }
    if (st == FEWHA_OK && geom->precision == FEWHA_F32) {
        h->work.reset(make_impl_f32(h->plan));
        st = h->work->init(geom->grid);
    } else if (st == FEWHA_OK && geom->precision == FEWHA_BF16S) {
        h->work.reset(make_impl_bf16(h->plan));
        st = h->work->init(geom->grid);
    }
    std::vector<double> invJ;
    if (st == FEWHA_OK) st = build_precond(*h, invJ);
    if (st == FEWHA_OK) st = h->f64->set_invJ(invJ);
    if (st == FEWHA_OK && h->work) st = h->work->set_invJ(invJ);
    if (st == FEWHA_OK && cudaDeviceSynchronize() != cudaSuccess) st = FEWHA_ERR_CUDA;
    if (st != FEWHA_OK) {
        delete h;
        return st;
    }
    *out = h;
    return FEWHA_OK;
}

void fewha_destroy(void *handle)
{
    if (!handle) return;
    cudaDeviceSynchronize();
    delete static_cast<Handle *>(handle);
}

long fewha_n_unknowns(const void *handle)
{
    return handle ? static_cast<const Handle *>(handle)->plan.n : -1;
}

long fewha_n_slopes(const void *handle)
{
    if (!handle) return -1;
    const Plan &p = static_cast<const Handle *>(handle)->plan;
    return 2L * p.ns * p.ns * p.G;
}

double fewha_layer_spacing(const void *handle, int layer)
{
    if (!handle) return -1.0;
    const Plan &p = static_cast<const Handle *>(handle)->plan;
    return (layer >= 0 && layer < p.L) ? p.lay_d[layer] : -1.0;
}

int fewha_get_prior(const void *handle, double *out)
{
    if (!handle || !out) return FEWHA_ERR_ARG;
    const Plan &p = static_cast<const Handle *>(handle)->plan;
    std::memcpy(out, p.alpha_d.data(), p.n * sizeof(double));
    return FEWHA_OK;
}

int fewha_get_precond(const void *handle, double *out)
{
    if (!handle || !out) return FEWHA_ERR_ARG;
    const Handle *h = static_cast<const Handle *>(handle);
    return h->work ? h->work->get_invJ(out) : h->f64->get_invJ(out);
}

// Vectors are accessed with 16-byte loads and stores.
static bool aligned16(const void *p) { return ((size_t)p & 15) == 0; }

int fewha_apply_op(void *handle, const void *x, void *y, cudaStream_t stream)
{
    if (!handle || !x || !y || x == y || !aligned16(x) || !aligned16(y)) return FEWHA_ERR_ARG;
    return static_cast<Handle *>(handle)->w()->apply(x, y, stream);
}

int fewha_rhs(void *handle, const void *s, void *b, cudaStream_t stream)
{
    if (!handle || !s || !b || !aligned16(b)) return FEWHA_ERR_ARG;
    return static_cast<Handle *>(handle)->w()->rhs(s, b, stream);
}

int fewha_solve(void *handle, const void *s, void *c, const fewha_state *st, const fewha_solve_opts *o,
                fewha_stats *stats, cudaStream_t stream)
{
    if (!handle || !s || !c || !st || !o) return FEWHA_ERR_ARG;
    if (!st->b_prev || !st->r_prev || !st->basis_P || !st->basis_Q || !st->basis_pq || !st->meta)
        return FEWHA_ERR_ARG;
    if (!aligned16(c) || !aligned16(st->b_prev) || !aligned16(st->r_prev) || !aligned16(st->basis_P) ||
        !aligned16(st->basis_Q))
        return FEWHA_ERR_ARG;
    if (st->k_cap < 1 || st->k_cap > FEWHA_MAX_K) return FEWHA_ERR_ARG;
    if (o->max_iter < 1 || o->max_iter > FEWHA_MAX_ITER || !(o->rtol >= 0)) return FEWHA_ERR_ARG;
    if (o->launch_mode != FEWHA_LAUNCH_PERSISTENT && o->launch_mode != FEWHA_LAUNCH_PHASES) return FEWHA_ERR_ARG;
    if (o->recycle_mode != FEWHA_RECYCLE_LAST && o->recycle_mode != FEWHA_RECYCLE_ALL) return FEWHA_ERR_ARG;
    return static_cast<Handle *>(handle)->w()->solve(s, c, st, o, stats, stream);
}

int fewha_set_timeout(void *handle, unsigned long long timeout_ns)
{
    if (!handle) return FEWHA_ERR_ARG;
    static_cast<Handle *>(handle)->w()->set_timeout(timeout_ns);
    return FEWHA_OK;
}

int fewha_set_trace(void *handle, unsigned long long *trace_dev, int capacity)
{
    if (!handle || (trace_dev && capacity < 1)) return FEWHA_ERR_ARG;
    static_cast<Handle *>(handle)->w()->set_trace(trace_dev, capacity);
    return FEWHA_OK;
}

const char *fewha_strerror(int status)
{
    switch (status) {
    case FEWHA_OK: return "ok";
    case FEWHA_ERR_ARG: return "invalid argument";
    case FEWHA_ERR_GEOMETRY: return "inconsistent geometry";
    case FEWHA_ERR_CUDA: return "CUDA runtime error";
    case FEWHA_ERR_TIMEOUT: return "device-side wait timed out";
    case FEWHA_ERR_BREAKDOWN: return "CG breakdown ((p, Mp) <= 0 or not finite)";
    case FEWHA_ERR_NOT_SPD: return "recycled Gram matrix not positive definite";
    case FEWHA_ERR_NOMEM: return "device allocation failed";
    case FEWHA_ERR_SCRATCH: return "problem too large for the fixed scratch of the allocation-free entry point";
    default: return "unknown status";
    }
}

}  // extern "C"
