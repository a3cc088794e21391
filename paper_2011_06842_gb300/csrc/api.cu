// libfewha: the C ABI (include/fewha.h) of the GB300 augmented FEWHA hot
// path.  The handle plans the geometry on the host, owns constant tables and
// scratch on the current device, and launches the kernels of one precision.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
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

// Vectors are accessed with 16-byte loads and stores.
static bool aligned16(const void *p) { return ((size_t)p & 15) == 0; }

const void *fewha_device_view(const void *p);  // transfer.cu

ImplBase *handle_impl(void *handle) { return handle ? static_cast<Handle *>(handle)->w() : nullptr; }
int handle_device(const void *handle) { return handle ? static_cast<const Handle *>(handle)->device : -1; }

// A batch: many instances (handles of one precision on one device) run by one
// cooperative launch, each by its own group of CTAs.
struct Batch {
    int n = 0, total = 0, nrounds = 1;  // total: CTAs of the launch (the largest round)
    size_t smem = 0, asz = 0;
    std::vector<ImplBase *> impl;
    std::vector<int> cta0, ncta, ty, tx;
    void *d_args = nullptr;
    void *d_bound = nullptr;  // argument table of fewha_batch_bind (fixed buffers, graph replay)
    bool bound = false;
    int bound_true_res = 0;  // the bound options ask for the residual replacement
    int *d_map = nullptr;                 // [nrounds][total] instance of each CTA, -1 idle
    Record *d_brec = nullptr;             // barrier between rounds
    static constexpr int kRing = 4;  // pinned staging copies of the argument table
    void *h_args[kRing] = {};
    cudaEvent_t ev[kRing] = {};
    int next = 0;
    ~Batch()
    {
        cudaFree(d_args);
        cudaFree(d_bound);
        cudaFree(d_map);
        cudaFree(d_brec);
        for (int i = 0; i < kRing; i++) {
            if (h_args[i]) cudaFreeHost(h_args[i]);
            if (ev[i]) cudaEventDestroy(ev[i]);
        }
    }
};

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
    // loads the module of fewha_apply_op_noalloc's static scratch on this
    // device now, while creating a handle may allocate (lazy module loading
    // would otherwise reserve it at the first allocation-free call)
    if (st == FEWHA_OK) st = noalloc_prepare();
    if (st == FEWHA_OK && cudaDeviceSynchronize() != cudaSuccess) st = FEWHA_ERR_CUDA;
    if (st != FEWHA_OK) {
        delete h;
        return st;
    }
    *out = h;
    return FEWHA_OK;
}

int fewha_set_noise(void *handle, const double *weight, int refresh_precond)
{
    if (!handle || !weight) return FEWHA_ERR_ARG;
    Handle *h = static_cast<Handle *>(handle);
    for (int g = 0; g < h->plan.G; g++)
        if (!std::isfinite(weight[g]) || !(weight[g] >= 0.0)) return FEWHA_ERR_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return FEWHA_ERR_CUDA;
    for (int g = 0; g < h->plan.G; g++) h->plan.geom.gs[g].weight = weight[g];
    int st = h->f64->set_weights();
    if (st == FEWHA_OK && h->work) st = h->work->set_weights();
    if (st == FEWHA_OK && refresh_precond) {
        std::vector<double> invJ;
        st = build_precond(*h, invJ);
        if (st == FEWHA_OK) st = h->f64->set_invJ(invJ);
        if (st == FEWHA_OK && h->work) st = h->work->set_invJ(invJ);
    }
    if (st == FEWHA_OK && cudaDeviceSynchronize() != cudaSuccess) st = FEWHA_ERR_CUDA;
    return st;
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
    return p.slope_off[p.G];
}

double fewha_layer_spacing(const void *handle, int layer)
{
    if (!handle) return -1.0;
    const Plan &p = static_cast<const Handle *>(handle)->plan;
    return (layer >= 0 && layer < p.L) ? p.lay_d[layer] : -1.0;
}

int fewha_get_launch_info(const void *handle, fewha_launch_info *out)
{
    if (!handle || !out) return FEWHA_ERR_ARG;
    const Handle *h = static_cast<const Handle *>(handle);
    (h->work ? h->work.get() : h->f64.get())->launch_info(out);
    return FEWHA_OK;
}

int fewha_set_pt_bands(void *handle, int rows_large, int rows_small)
{
    if (!handle || rows_large < 1 || rows_small < 1) return FEWHA_ERR_ARG;
    Handle *h = static_cast<Handle *>(handle);
    if (cudaSetDevice(h->device) != cudaSuccess) return FEWHA_ERR_CUDA;
    return h->w()->set_bands(rows_large, rows_small);
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

int fewha_apply_op(void *handle, const void *x, void *y, cudaStream_t stream)
{
    if (!handle || !x || !y || x == y || !aligned16(x) || !aligned16(y)) return FEWHA_ERR_ARG;
    return static_cast<Handle *>(handle)->w()->apply(x, y, stream);
}

int fewha_apply_op_multi(void *handle, const void *x, long ldx, void *y, long ldy, int nvec, cudaStream_t stream)
{
    if (!handle || !x || !y || nvec < 1 || nvec > FEWHA_MAX_MULTI || !aligned16(x) || !aligned16(y)) return FEWHA_ERR_ARG;
    Handle *h = static_cast<Handle *>(handle);
    const long n = h->plan.n;
    if (ldx < n || ldy < n || (ldx % 4) || (ldy % 4)) return FEWHA_ERR_ARG;
    const size_t es = h->w()->precision_id() == FEWHA_F64 ? 8 : 4;
    const char *xb = static_cast<const char *>(x), *yb = static_cast<const char *>(y);
    const char *xe = xb + ((nvec - 1) * ldx + n) * es, *ye = yb + ((nvec - 1) * ldy + n) * es;
    if (xb < ye && yb < xe) return FEWHA_ERR_ARG;  // x and y must not overlap
    return h->w()->apply_multi(x, ldx, y, ldy, nvec, stream);
}

long fewha_n_actuators(const void *handle)
{
    if (!handle) return -1;
    const long m = static_cast<const Handle *>(handle)->plan.m;
    return m * m;
}

int fewha_fit(void *handle, const void *c, void *a_fit, cudaStream_t stream)
{
    if (!handle || !c || !a_fit || !aligned16(c)) return FEWHA_ERR_ARG;
    return static_cast<Handle *>(handle)->w()->fit(c, a_fit, stream);
}

// MCAO fitting object: the handle's working-precision implementation and its plan
struct Mcao {
    ImplBase *impl = nullptr;
    int device = 0;
    void *plan = nullptr;
    long n_act = 0;
};

int fewha_mcao_create(void *handle, const fewha_mcao_desc *desc, void **mcao_out)
{
    if (!handle || !desc || !mcao_out) return FEWHA_ERR_ARG;
    *mcao_out = nullptr;
    Handle *h = static_cast<Handle *>(handle);
    if (cudaSetDevice(h->device) != cudaSuccess) return FEWHA_ERR_CUDA;
    auto *m = new Mcao();
    m->impl = h->w();
    m->device = h->device;
    const int st = m->impl->mcao_create(desc, &m->plan, &m->n_act);
    if (st) {
        delete m;
        return st;
    }
    *mcao_out = m;
    return FEWHA_OK;
}

long fewha_mcao_n_actuators(const void *mcao) { return mcao ? static_cast<const Mcao *>(mcao)->n_act : -1; }

int fewha_mcao_fit(void *mcao, const void *c, void *a, int iters, cudaStream_t stream)
{
    if (!mcao || !c || !a || !aligned16(c)) return FEWHA_ERR_ARG;
    Mcao *m = static_cast<Mcao *>(mcao);
    return m->impl->mcao_fit(m->plan, c, a, iters, stream);
}

void fewha_mcao_destroy(void *mcao)
{
    if (!mcao) return;
    Mcao *m = static_cast<Mcao *>(mcao);
    cudaSetDevice(m->device);
    if (m->plan) m->impl->mcao_destroy(m->plan);
    delete m;
}

int fewha_pol_slopes(void *handle, const void *s, const void *a_prev, void *s_out, cudaStream_t stream)
{
    if (!handle || !s || !a_prev || !s_out) return FEWHA_ERR_ARG;
    return static_cast<Handle *>(handle)->w()->pol_slopes(s, a_prev, s_out, stream);
}

int fewha_control(void *handle, int closed, double gain, const void *a_im1, const void *a_i, const void *a_fit,
                  void *a_next, cudaStream_t stream)
{
    if (!handle || !a_im1 || !a_i || !a_fit || !a_next || !(gain >= 0.0 && gain <= 1.0)) return FEWHA_ERR_ARG;
    return static_cast<Handle *>(handle)->w()->control(closed ? 1 : 0, gain, a_im1, a_i, a_fit, a_next, stream);
}

int fewha_rhs(void *handle, const void *s, void *b, cudaStream_t stream)
{
    if (!handle || !s || !b || !aligned16(b)) return FEWHA_ERR_ARG;
    s = fewha_device_view(s);  // device, managed or page-locked host slopes
    if (!s) return FEWHA_ERR_ARG;
    return static_cast<Handle *>(handle)->w()->rhs(s, b, stream);
}

int fewha_solve(void *handle, const void *s, void *c, const fewha_state *st, const fewha_solve_opts *o,
                fewha_stats *stats, cudaStream_t stream)
{
    if (!handle || !c || !st || !o || (!s && !o->rhs_in_state)) return FEWHA_ERR_ARG;
    if (!st->b_prev || !st->r_prev || !st->basis_P || !st->basis_Q || !st->basis_pq || !st->meta)
        return FEWHA_ERR_ARG;
    if (!aligned16(c) || !aligned16(st->b_prev) || !aligned16(st->r_prev) || !aligned16(st->basis_P) ||
        !aligned16(st->basis_Q))
        return FEWHA_ERR_ARG;
    if (st->k_cap < 1 || st->k_cap > FEWHA_MAX_K) return FEWHA_ERR_ARG;
    if (o->max_iter < 1 || o->max_iter > FEWHA_MAX_ITER || !(o->rtol >= 0)) return FEWHA_ERR_ARG;
    if (o->true_res_every < 0 || o->true_res_every > FEWHA_MAX_ITER) return FEWHA_ERR_ARG;
    if (o->launch_mode != FEWHA_LAUNCH_PERSISTENT && o->launch_mode != FEWHA_LAUNCH_PHASES) return FEWHA_ERR_ARG;
    if (o->recycle_mode != FEWHA_RECYCLE_LAST && o->recycle_mode != FEWHA_RECYCLE_ALL) return FEWHA_ERR_ARG;
    if (!o->rhs_in_state) {
        s = fewha_device_view(s);  // device, managed or page-locked host slopes
        if (!s) return FEWHA_ERR_ARG;
    }
    fewha_solve_opts ov = *o;
    if (ov.c_out) {
        // the second destination of the solution, as the device reaches it
        Handle *h = static_cast<Handle *>(handle);
        const size_t bytes = (size_t)h->plan.n * (h->w()->precision_id() == FEWHA_F64 ? 8 : 4);
        ov.c_out = const_cast<void *>(fewha_device_view(o->c_out));
        if (!ov.c_out || !aligned16(ov.c_out)) return FEWHA_ERR_ARG;
        const char *a = static_cast<const char *>(ov.c_out), *cc = static_cast<const char *>(c);
        if (a < cc + bytes && cc < a + bytes) return FEWHA_ERR_ARG;  // must not overlap c
    }
    return static_cast<Handle *>(handle)->w()->solve(s, c, st, &ov, stats, stream);
}

int fewha_batch_create(void *const *handles, int n, const int *ctas, void **batch_out)
{
    return fewha_batch_create_rounds(handles, n, ctas, nullptr, batch_out);
}

int fewha_batch_create_rounds(void *const *handles, int n, const int *ctas, const int *rounds, void **batch_out)
{
    return fewha_batch_create_ex(handles, n, ctas, rounds, nullptr, batch_out);
}

int fewha_batch_create_ex(void *const *handles, int n, const int *ctas, const int *rounds, const int *tiles,
                          void **batch_out)
{
    if (!handles || n < 1 || !batch_out) return FEWHA_ERR_ARG;
    *batch_out = nullptr;
    std::unique_ptr<Batch> b(new (std::nothrow) Batch());
    if (!b) return FEWHA_ERR_NOMEM;
    b->n = n;
    int prec = -1;
    std::vector<double> weight(n);
    std::vector<int> round(n, 0);
    for (int i = 0; i < n; i++) {
        if (!handles[i]) return FEWHA_ERR_ARG;
        Handle *h = static_cast<Handle *>(handles[i]);
        b->impl.push_back(h->w());
        if (prec >= 0 && h->w()->precision_id() != prec) return FEWHA_ERR_ARG;
        prec = h->w()->precision_id();
        // work of one iteration ~ unknowns + adjoint wavefront nodes
        weight[i] = (double)h->plan.n + (double)h->plan.G * h->plan.m * h->plan.m;
        if (rounds) {
            if (rounds[i] < 0 || rounds[i] >= n) return FEWHA_ERR_ARG;
            round[i] = rounds[i];
        }
    }
    b->nrounds = 1 + *std::max_element(round.begin(), round.end());
    // CTA groups: given, or per round proportional to the work (at least one each)
    int cap = 0;
    int st = b->impl[0]->batch_capacity(200 * 1024, &cap);
    if (st) return st;
    b->ncta.assign(n, 1);
    if (ctas) {
        for (int i = 0; i < n; i++) {
            if (ctas[i] < 1) return FEWHA_ERR_ARG;
            b->ncta[i] = ctas[i];
        }
    } else {
        for (int r = 0; r < b->nrounds; r++) {
            int nr = 0;
            double wsum = 0;
            for (int i = 0; i < n; i++)
                if (round[i] == r) nr++, wsum += weight[i];
            if (nr == 0) continue;
            if (nr > cap) return FEWHA_ERR_ARG;
            int used = 0;
            for (int i = 0; i < n; i++)
                if (round[i] == r) {
                    b->ncta[i] = std::max(1, (int)((cap - nr) * weight[i] / wsum) + 1);
                    used += b->ncta[i];
                }
            while (used > cap) {  // trim the largest groups of the round
                int j = -1;
                for (int i = 0; i < n; i++)
                    if (round[i] == r && (j < 0 || b->ncta[i] > b->ncta[j])) j = i;
                b->ncta[j]--;
                used--;
            }
        }
    }
    b->cta0.resize(n);
    b->ty.resize(n);
    b->tx.resize(n);
    std::vector<int> used(b->nrounds, 0);
    for (int i = 0; i < n; i++) {
        b->cta0[i] = used[round[i]];
        used[round[i]] += b->ncta[i];
        if (tiles && (tiles[2 * i] || tiles[2 * i + 1])) {
            b->ty[i] = tiles[2 * i];
            b->tx[i] = tiles[2 * i + 1];
            if (b->ty[i] < 4 || b->ty[i] > 64 || b->tx[i] < 4 || b->tx[i] > 64 ||
                b->impl[i]->smem_for(b->ty[i], b->tx[i]) > 200 * 1024)
                return FEWHA_ERR_ARG;
        } else if ((st = b->impl[i]->tiles_for(b->ncta[i], &b->ty[i], &b->tx[i]))) {
            return st;
        }
        b->smem = std::max(b->smem, b->impl[i]->smem_for(b->ty[i], b->tx[i]));
    }
    b->total = *std::max_element(used.begin(), used.end());
    if ((st = b->impl[0]->batch_capacity(b->smem, &cap))) return st;
    if (b->total > cap) return FEWHA_ERR_ARG;  // every round's groups must be co-resident
    b->asz = b->impl[0]->args_size();
    std::vector<int> map((size_t)b->nrounds * b->total, -1);
    for (int i = 0; i < n; i++)
        for (int c = 0; c < b->ncta[i]; c++) map[(size_t)round[i] * b->total + b->cta0[i] + c] = i;
    if (cudaMalloc(&b->d_args, b->asz * n) != cudaSuccess ||
        cudaMalloc(&b->d_map, sizeof(int) * map.size()) != cudaSuccess ||
        cudaMalloc(&b->d_brec, sizeof(Record)) != cudaSuccess)
        return FEWHA_ERR_NOMEM;
    if (cudaMemcpy(b->d_map, map.data(), sizeof(int) * map.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_brec, 0, sizeof(Record)) != cudaSuccess)
        return FEWHA_ERR_CUDA;
    for (int i = 0; i < Batch::kRing; i++) {
        if (cudaHostAlloc(&b->h_args[i], b->asz * n, cudaHostAllocDefault) != cudaSuccess) return FEWHA_ERR_NOMEM;
        if (cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming) != cudaSuccess) return FEWHA_ERR_CUDA;
    }
    *batch_out = b.release();
    return FEWHA_OK;
}

int fewha_batch_ctas(const void *batch, int *ctas_out)
{
    if (!batch || !ctas_out) return FEWHA_ERR_ARG;
    const Batch *b = static_cast<const Batch *>(batch);
    for (int i = 0; i < b->n; i++) ctas_out[i] = b->ncta[i];
    return FEWHA_OK;
}

int fewha_batch_tiles(const void *batch, int *tiles_out)
{
    if (!batch || !tiles_out) return FEWHA_ERR_ARG;
    const Batch *b = static_cast<const Batch *>(batch);
    for (int i = 0; i < b->n; i++) {
        tiles_out[2 * i] = b->ty[i];
        tiles_out[2 * i + 1] = b->tx[i];
    }
    return FEWHA_OK;
}

int fewha_batch_solve(void *batch, const void *const *slopes, void *const *c, const fewha_state *states,
                      const fewha_solve_opts *opts, fewha_stats *stats_dev, cudaStream_t stream)
{
    if (!batch || !slopes || !c || !states || !opts) return FEWHA_ERR_ARG;
    Batch *b = static_cast<Batch *>(batch);
    if (opts->max_iter < 1 || opts->max_iter > FEWHA_MAX_ITER || !(opts->rtol >= 0)) return FEWHA_ERR_ARG;
    if (opts->true_res_every < 0 || opts->true_res_every > FEWHA_MAX_ITER) return FEWHA_ERR_ARG;
    if (opts->rhs_in_state) return FEWHA_ERR_ARG;  // batches form their right-hand sides
    if (opts->recycle_mode != FEWHA_RECYCLE_LAST && opts->recycle_mode != FEWHA_RECYCLE_ALL) return FEWHA_ERR_ARG;
    const int slot = b->next;
    b->next = (b->next + 1) % Batch::kRing;
    if (cudaEventSynchronize(b->ev[slot]) != cudaSuccess) return FEWHA_ERR_CUDA;  // staging copy free again
    unsigned char *h = static_cast<unsigned char *>(b->h_args[slot]);
    for (int i = 0; i < b->n; i++) {
        const fewha_state *st = states + i;
        if (!slopes[i] || !c[i] || !st->b_prev || !st->r_prev || !st->basis_P || !st->basis_Q || !st->basis_pq ||
            !st->meta || st->k_cap < 1 || st->k_cap > FEWHA_MAX_K)
            return FEWHA_ERR_ARG;
        if (b->impl[i]->smem_for(b->ty[i], b->tx[i]) > b->smem) return FEWHA_ERR_ARG;  // re-planned since
        if (!aligned16(c[i]) || !aligned16(st->b_prev) || !aligned16(st->r_prev) || !aligned16(st->basis_P) ||
            !aligned16(st->basis_Q))
            return FEWHA_ERR_ARG;
        int r = b->impl[i]->batch_args(h + b->asz * i, slopes[i], c[i], st, opts, stats_dev ? stats_dev + i : nullptr,
                                       b->cta0[i], b->ncta[i], b->ty[i], b->tx[i], b->smem);
        if (r) return r;
    }
    if (cudaMemcpyAsync(b->d_args, h, b->asz * b->n, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return FEWHA_ERR_CUDA;
    if (cudaEventRecord(b->ev[slot], stream) != cudaSuccess) return FEWHA_ERR_CUDA;
    return b->impl[0]->launch_batched(b->d_args, b->d_map, b->n, b->total, b->smem, b->nrounds, b->d_brec,
                                      opts->true_res_every > 0, stream);
}

int fewha_batch_bind(void *batch, const void *const *slopes, void *const *c, const fewha_state *states,
                     const fewha_solve_opts *opts, fewha_stats *stats_dev)
{
    if (!batch || !slopes || !c || !states || !opts) return FEWHA_ERR_ARG;
    Batch *b = static_cast<Batch *>(batch);
    if (opts->max_iter < 1 || opts->max_iter > FEWHA_MAX_ITER || !(opts->rtol >= 0)) return FEWHA_ERR_ARG;
    if (opts->true_res_every < 0 || opts->true_res_every > FEWHA_MAX_ITER) return FEWHA_ERR_ARG;
    if (opts->rhs_in_state) return FEWHA_ERR_ARG;  // batches form their right-hand sides
    if (opts->recycle_mode != FEWHA_RECYCLE_LAST && opts->recycle_mode != FEWHA_RECYCLE_ALL) return FEWHA_ERR_ARG;
    std::vector<unsigned char> h(b->asz * b->n);
    for (int i = 0; i < b->n; i++) {
        const fewha_state *st = states + i;
        if (!slopes[i] || !c[i] || !st->b_prev || !st->r_prev || !st->basis_P || !st->basis_Q || !st->basis_pq ||
            !st->meta || st->k_cap < 1 || st->k_cap > FEWHA_MAX_K)
            return FEWHA_ERR_ARG;
        if (b->impl[i]->smem_for(b->ty[i], b->tx[i]) > b->smem) return FEWHA_ERR_ARG;  // re-planned since
        if (!aligned16(c[i]) || !aligned16(st->b_prev) || !aligned16(st->r_prev) || !aligned16(st->basis_P) ||
            !aligned16(st->basis_Q))
            return FEWHA_ERR_ARG;
        int r = b->impl[i]->batch_args(h.data() + b->asz * i, slopes[i], c[i], st, opts,
                                       stats_dev ? stats_dev + i : nullptr, b->cta0[i], b->ncta[i], b->ty[i], b->tx[i],
                                       b->smem);
        if (r) return r;
    }
    if (!b->d_bound && cudaMalloc(&b->d_bound, b->asz * b->n) != cudaSuccess) return FEWHA_ERR_NOMEM;
    if (cudaMemcpy(b->d_bound, h.data(), b->asz * b->n, cudaMemcpyHostToDevice) != cudaSuccess) return FEWHA_ERR_CUDA;
    b->bound = true;
    b->bound_true_res = opts->true_res_every > 0;
    return FEWHA_OK;
}

int fewha_batch_launch(void *batch, cudaStream_t stream)
{
    if (!batch) return FEWHA_ERR_ARG;
    Batch *b = static_cast<Batch *>(batch);
    if (!b->bound) return FEWHA_ERR_ARG;
    for (int i = 0; i < b->n; i++)
        if (b->impl[i]->smem_for(b->ty[i], b->tx[i]) > b->smem) return FEWHA_ERR_ARG;  // re-planned since
    return b->impl[0]->launch_batched(b->d_bound, b->d_map, b->n, b->total, b->smem, b->nrounds, b->d_brec,
                                      b->bound_true_res, stream);
}

void fewha_batch_destroy(void *batch)
{
    if (!batch) return;
    cudaDeviceSynchronize();
    delete static_cast<Batch *>(batch);
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
