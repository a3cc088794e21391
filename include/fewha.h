/*
 * fewha.h - C ABI of the GB300 (sm_103a) augmented-FEWHA tomography library.
 *
 * The library applies the FEWHA normal operator
 *     M = W^{-T} A^T C_eta^{-1} A W^{-1} + alpha D            (Ramlau & Stadler, Sec. 3, Eq. M)
 * matrix-free on the GPU and solves M c = b with preconditioned CG
 * (Algorithm 1) or augmented, Krylov-recycled PCG (Algorithm 2) inside one
 * time step of the reconstructor loop (Algorithm 3: right-hand side, warm
 * restart residual, solve).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Status: every function returns 0 (FEWHA_OK) or a negative FEWHA_ERR_*
 *    code; nothing throws across the ABI.  Errors raised on the device
 *    (barrier timeout, CG breakdown) are reported in fewha_stats.status,
 *    valid after the stream has been synchronised.
 *  - Memory: all vectors passed to the compute calls are DEVICE pointers owned
 *    by the caller, allocated on the device the handle was created on; the
 *    slopes of fewha_rhs / fewha_solve may also be page-locked host memory
 *    (read in place by the kernels), and fewha_store may write to it.
 *    Coefficient vectors (x, y, b, c and the state vectors) must be 16-byte
 *    aligned (FEWHA_ERR_ARG otherwise); slopes need only element alignment.  The
 *    handle owns its constant tables and its scratch memory.  Nothing is
 *    retained after a call returns except the handle's own state.
 *  - Element type of the vectors: double for FEWHA_F64 handles, float for
 *    FEWHA_F32 and FEWHA_BF16S handles.  Slopes are double / float /
 *    bfloat16 (raw 16-bit, round-to-nearest-even) respectively.
 *  - Layout of a coefficient vector c (length n = sum_l n_l^2): layer after
 *    layer; inside a layer the n_l x n_l array of periodic Daubechies wavelet
 *    coefficients in row-major Mallat layout (coarsest approximation block in
 *    the top-left corner; at every level the block right of it is low-pass in
 *    y and high-pass in x, the block below high-pass in y and low-pass in x).
 *  - Layout of a slope vector s (length sum_g 2 n_g^2, n_g the subapertures
 *    across guide star g's sensor): guide star after guide star, each
 *    [x slopes | y slopes], each n_g x n_g row-major (row = y).  Entries of
 *    unlit subapertures are ignored.
 *  - Asynchrony: compute calls enqueue work on the given stream and return.
 */
#ifndef FEWHA_H
#define FEWHA_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *cudaStream_t;

#define FEWHA_MAX_GS 16
#define FEWHA_MAX_LAYERS 16
#define FEWHA_MAX_K 16        /* largest recycled basis */
#define FEWHA_MAX_ITER 1000   /* largest max_iter of one solve */
#define FEWHA_MAX_GRID 128    /* largest layer grid (n_l); the layer must fit one SM's shared memory */

enum {
    FEWHA_OK = 0,
    FEWHA_ERR_ARG = -1,       /* bad pointer, size or option */
    FEWHA_ERR_GEOMETRY = -2,  /* inconsistent telescope / layer geometry */
    FEWHA_ERR_CUDA = -3,      /* a CUDA runtime call failed */
    FEWHA_ERR_TIMEOUT = -4,   /* a device-side wait gave up (grid barrier) */
    FEWHA_ERR_BREAKDOWN = -5, /* CG breakdown: (p, Mp) <= 0 or not finite */
    FEWHA_ERR_NOT_SPD = -6,   /* recycled Gram matrix not positive definite */
    FEWHA_ERR_NOMEM = -7,     /* device allocation failed */
    FEWHA_ERR_SCRATCH = -8    /* problem too large for fewha_apply_op_noalloc's fixed scratch */
};

enum { FEWHA_F64 = 0, FEWHA_F32 = 1, FEWHA_BF16S = 2 };

/* Guide star (Sec. 2): direction theta [rad]; H = sodium-layer height [m] for
 * a laser guide star (cone effect, P^LGS), H <= 0 for a natural guide star
 * (P^NGS); weight = 1/sigma^2, the diagonal of C_eta^{-1} on its lit
 * subapertures (Sec. 3); n_sub = subapertures across its Shack-Hartmann
 * sensor (0: the geometry's n_sub), so that low-order sensors (the MCAO
 * asterism's 2x2 and 1x1 NGS, Sec. 5.1) sit beside high-order ones.  Every
 * sensor spans the pupil: sensor g has (n_g+1)^2 pupil nodes at spacing
 * D / n_g; a subaperture is lit iff its centre radius lies in
 * [obstruction D/2, D/2], and the single subaperture of a 1x1 sensor is
 * always lit. */
typedef struct {
    double theta_x, theta_y, H, weight;
    int n_sub;
    int pad;
} fewha_gs;

/* Turbulent layer (Sec. 2, Eq. atmo): height h [m], Cn2 fraction (prior D),
 * node grid n x n (power of two, 8..FEWHA_MAX_GRID), J wavelet levels
 * (n >> J >= 1), scaling constant delta of W = diag(delta_l W) (Eq. fewha). */
typedef struct {
    double h, cn2, delta;
    int n, J;
} fewha_layer;

/* Telescope, sensors and layers (Sec. 2, Sec. 5.1 parameter table). */
typedef struct {
    double D;             /* pupil diameter [m] */
    double obstruction;   /* central obstruction, fraction of D */
    int n_sub;            /* Shack-Hartmann subapertures across the pupil (n_s) */
    int n_gs;
    fewha_gs gs[FEWHA_MAX_GS];
    int n_layers;
    fewha_layer layers[FEWHA_MAX_LAYERS];
    double r0;            /* Fried parameter [m] of the prior D */
    double alpha;         /* regularisation weight alpha of Eq. fewha */
    int wavelet_N;        /* Daubechies vanishing moments (3 = Daubechies-3, 6 taps), 1..4 */
    int precision;        /* FEWHA_F64, FEWHA_F32 or FEWHA_BF16S */
    int tile;             /* WFS tile edge in pupil nodes (8, 16 or 32); 0 = default */
    int grid;             /* CTAs of the solver launch; 0 = one per SM */
} fewha_geometry;

/* Per-time-step solver state (Algorithm 3 inputs and outputs), caller-owned
 * device memory of the handle's vector type:
 *   b_prev[n], r_prev[n]   previous right-hand side and residual (zero at frame 0);
 *   basis_P[2*k_cap*n], basis_Q[2*k_cap*n]   two banks of recycled directions
 *                          p and q = M p (the solve reads one bank, writes the other);
 *   basis_pq[2*k_cap]      (p_j, q_j) in double;
 *   meta[4]                ints: active bank, directions in it, newest slot,
 *                          frames solved (all zero at frame 0). */
typedef struct {
    void *b_prev, *r_prev, *basis_P, *basis_Q;
    double *basis_pq;
    int *meta;
    int k_cap;            /* 1..FEWHA_MAX_K */
} fewha_state;

enum { FEWHA_RECYCLE_LAST = 0, FEWHA_RECYCLE_ALL = 1 };
enum { FEWHA_LAUNCH_PERSISTENT = 0, FEWHA_LAUNCH_PHASES = 1 };

typedef struct {
    int max_iter;         /* iterations k = 0..max_iter-1 (1..FEWHA_MAX_ITER) */
    double rtol;          /* > 0: stop once ||r|| <= rtol ||b|| (recurrence residual) */
    int augmented;        /* 0: PCG (Algorithm 1); 1: augmented PCG (Algorithm 2) */
    int recycle_mode;     /* FEWHA_RECYCLE_LAST (paper) or FEWHA_RECYCLE_ALL */
    int launch_mode;      /* FEWHA_LAUNCH_PERSISTENT (one kernel) or FEWHA_LAUNCH_PHASES */
    /* N > 0: residual replacement.  After iterations N, 2N, 3N, ... (counting
     * from 1) the recurrence residual r is replaced by the true residual
     * b - M c, computed with one more operator application whose
     * intermediates are stored in the working precision (FP32 also for
     * FEWHA_BF16S); z = J^{-1} r, the projection, (r, z) and beta of the next
     * iteration, the stopping test and the next time step's warm restart
     * then see the true residual.  0 = off (the paper: Algorithms 1-3 keep
     * the recurrence residual).  0..FEWHA_MAX_ITER. */
    int true_res_every;
    /* 1: this time step's right-hand side is already folded into the state
     * (b_prev = b, r_prev = the warm-restart residual r0), as
     * fewha_deflate_warm_start leaves it: the solve skips the right-hand-side
     * phases and does not read the slopes (s may be NULL).  0: Algorithm 3's
     * right-hand side and warm restart from s. */
    int rhs_in_state;
    int pad;
    /* Optional (NULL: none): at the end of the time step the solution c is
     * also written here by the solve kernel itself: device, managed or
     * page-locked host memory (n elements of c's type, 16-byte aligned, not
     * overlapping c); pageable host memory is refused (FEWHA_ERR_ARG).  With
     * page-locked host memory the solution reaches the host with no transfer
     * on the stream.  Ignored by the batch calls. */
    void *c_out;
} fewha_solve_opts;

/* Written on the device at the end of fewha_solve. */
typedef struct {
    int status;           /* FEWHA_OK or a device-side FEWHA_ERR_* */
    int iterations;       /* PCG iterations run */
    double rel_res;       /* ||r|| / ||b|| of the recurrence residual at exit */
    double bnorm;         /* ||b|| */
    double rz;            /* (r, z) at exit */
    int basis_count;      /* recycled directions available to the next frame */
    int pad;
} fewha_stats;

/* Builds the operator for one geometry (Sec. 2-4): layer grids, interpolation
 * tables of P_g, subaperture mask, prior D, Daubechies taps, and the modified
 * Jacobi preconditioner J (computed on the GPU in FP64 from sampled diagonal
 * entries of M).  Uses the current CUDA device.  Blocking. */
int fewha_create(const fewha_geometry *geom, void **handle_out);

/* Noise weights C_eta^{-1} (Sec. 3, Eq. M: the diagonal of C_eta^{-1} is
 * weight[g] = 1/sigma_g^2 on the lit subapertures of guide star g, 0
 * elsewhere), for g = 0..n_gs-1: finite and >= 0 (FEWHA_ERR_ARG otherwise).
 * Replaces the weights given at fewha_create in the operator M and the
 * right-hand side of every later call.  The modified Jacobi preconditioner J
 * (Sec. 4) depends on them through its data term: with refresh_precond != 0
 * it is rebuilt from sampled diagonal entries of the new M (the same
 * FP64 sampling as fewha_create, several hundred operator applications);
 * with 0 it keeps the values computed for the earlier weights (still a valid
 * SPD preconditioner, only less well matched).  Waits for the device to be
 * idle before it writes the tables and again at the end (blocking): call it
 * between time steps, never while a solve on this handle is in flight. */
int fewha_set_noise(void *handle, const double *weight, int refresh_precond);

/* Frees the handle and its device memory (synchronises the device). */
void fewha_destroy(void *handle);

/* n (unknowns), slopes (sum_g 2 n_g^2), and the layer spacing d_l [m]. */
long fewha_n_unknowns(const void *handle);
long fewha_n_slopes(const void *handle);
double fewha_layer_spacing(const void *handle, int layer);

/* Launch shape of the handle's single-instance kernels (working precision),
 * as chosen at creation for the current GPU: CTAs (one per SM unless the
 * geometry's `grid` fixed them), threads per CTA, dynamic shared memory, and
 * which forms of the operator phases run: split_levels = 1 when the finest
 * wavelet level is tiled over all CTAs and only the coarser levels stay on
 * one CTA per layer (at least twice as many CTAs as layers), 0 when each
 * layer's CTA runs every level; staged_tables = 1 when the P_g^T gather
 * stages its interpolation-weight tables in shared memory beside the adjoint
 * wavefront rows, 0 when it reads them from global memory; the WFS tile
 * shape; the P_g^T work items (bands of layer rows) and the adjoint wavefront
 * rows staged per pass.  Host only, no device work.  The paper has no
 * counterpart. */
typedef struct {
    int ctas, threads;
    long smem_bytes;
    int split_levels, staged_tables;
    int wfs_tile_y, wfs_tile_x;
    int pt_bands, pt_rows_chunk;
    int pt_rows_large, pt_rows_small;  /* P^T band height on the largest / the smaller layers */
} fewha_launch_info;
int fewha_get_launch_info(const void *handle, fewha_launch_info *out);

/* Height of the P_g^T gather's work items (bands of layer rows): rows_large
 * on the layers of the largest grid, rows_small on the smaller ones (default
 * 8 and 4); each is capped so that a band has at most 1024 layer nodes.
 * Re-plans the band tables and the shared memory they need; FEWHA_ERR_GEOMETRY
 * (and the earlier plan kept) when the staged rows do not fit.  Waits for the
 * device to be idle (blocking); batches created before the call are refused
 * by fewha_batch_solve / fewha_batch_bind when their shared memory no longer
 * suffices.  A tuning knob (fewha autotuner); results do not depend on it
 * beyond rounding order.  The paper has no counterpart. */
int fewha_set_pt_bands(void *handle, int rows_large, int rows_small);

/* Copies the diagonal of alpha*D (Sec. 3) or of J^{-1} (Sec. 4) to host memory (n doubles). */
int fewha_get_prior(const void *handle, double *alpha_d_host);
int fewha_get_precond(const void *handle, double *invJ_host);

/* y = M x (Eq. M).  x, y: device vectors of length n; must not overlap. */
int fewha_apply_op(void *handle, const void *x, void *y, cudaStream_t stream);

/* y_v = M x_v for v = 0..nvec-1 (x_v = x + v*ldx, y_v = y + v*ldy elements,
 * 1 <= nvec <= FEWHA_MAX_MULTI, ld >= n and a multiple of 4; x and y must not
 * overlap).  One launch per operator stage for all vectors, each vector on
 * its own share of the CTAs (used for the directions of a deflated warm start). */
#define FEWHA_MAX_MULTI 8
int fewha_apply_op_multi(void *handle, const void *x, long ldx, void *y, long ldy, int nvec, cudaStream_t stream);

/* b = W^{-T} A^T C_eta^{-1} s (right-hand side of Eq. fewha; Algorithm 3).
 * s: device, managed or page-locked host memory (cudaHostAlloc,
 * cudaMallocHost, cudaHostRegister), read by the kernels where it lies;
 * pageable host memory is refused (FEWHA_ERR_ARG). */
int fewha_rhs(void *handle, const void *s, void *b, cudaStream_t stream);

/* Mirror side of the reconstructor loop (Algorithm 3).  Reading of the
 * fitting operator F, which the paper names but does not write out: one
 * deformable mirror conjugated to the ground whose actuators sit on the
 * (n_s+1)^2 pupil nodes (the subaperture corners, Fried geometry); the phase it
 * adds at a pupil node is the actuator value there, the same for every guide
 * star.  Mirror vectors (n_actuators, row-major (n_s+1) x (n_s+1)) are device
 * arrays of the working precision's vector type (double for FEWHA_F64, float
 * otherwise); slopes use the slope type of fewha_solve.
 *
 * fewha_n_actuators: (n_s+1)^2.
 * fewha_fit: a_fit = F W^{-1} c, the on-axis projection (direction 0, no cone)
 *   of every layer onto the actuators, bilinear on each layer grid (the
 *   fitting step of Algorithm 3).  FEWHA_ERR_GEOMETRY if an actuator projects
 *   outside a layer grid.  c 16-byte aligned.
 * fewha_pol_slopes: s_out = s + Gamma a_prev for every guide star (the
 *   pseudo-open-loop measurements of a closed loop; a_prev is the mirror shape
 *   applied two steps earlier).  s_out may equal s.  The mirror's actuators
 *   sit on the geometry's pupil grid, so every sensor must have the
 *   geometry's n_sub (FEWHA_ERR_GEOMETRY otherwise).
 * fewha_control: closed != 0: a_next = a_i + gain (a_fit - a_{i-1}); closed ==
 *   0: a_next = (1 - gain) a_i + gain a_fit (gain control); 0 <= gain <= 1.
 * All asynchronous on `stream`; FEWHA_ERR_ARG for NULL handles or pointers. */
long fewha_n_actuators(const void *handle);
int fewha_fit(void *handle, const void *c, void *a_fit, cudaStream_t stream);
int fewha_pol_slopes(void *handle, const void *s, const void *a_prev, void *s_out, cudaStream_t stream);
int fewha_control(void *handle, int closed, double gain, const void *a_im1, const void *a_i, const void *a_fit,
                  void *a_next, cudaStream_t stream);

/* One reconstructor time step (Algorithm 3, RHS to augPCG):
 *   b = rhs(s); r0 = (b - b_prev) + r_prev; b_prev <- b;
 *   (aug)PCG from the warm start c, updating c (in/out, device, n) and r_prev;
 *   the directions of this solve become the recycled basis of the next one.
 * s: as for fewha_rhs (device, managed or page-locked host memory: a frame's
 * slopes can be read by the kernel straight from the page-locked buffer the
 * sensors write, with no copy on the stream); pageable host memory is refused.
 * stats_dev: device pointer to a fewha_stats, written at the end. */
int fewha_solve(void *handle, const void *s, void *c, const fewha_state *state,
                const fewha_solve_opts *opts, fewha_stats *stats_dev, cudaStream_t stream);

/* Batched time steps: n instances (handles of one precision, on the current
 * device, geometries may differ) solved by ONE cooperative launch, each by its
 * own group of CTAs with its own barrier, reductions and recycled basis.
 * ctas: CTAs per instance (NULL: proportional to the work of one iteration,
 * n_l^2 summed over layers plus G (n_s+1)^2, at least one each); the groups
 * must fit the GPU at once (FEWHA_ERR_ARG otherwise).  The WFS tile shape of
 * every instance is re-chosen for its group.  fewha_batch_solve takes one
 * pointer per instance (slopes, c, state; stats_dev: n consecutive records)
 * and the same options for all; it stages the launch arguments through a
 * small ring of pinned host buffers, so it can be captured in a CUDA graph
 * (the graph then replays the captured pointers).  Blocking only when all
 * four staging buffers are still in flight.  Not in the paper: the paper
 * solves one system per time step. */
int fewha_batch_create(void *const *handles, int n, const int *ctas, void **batch_out);
/* Same, with the instances in rounds: rounds[i] (0, 1, ...) is the round of
 * instance i (NULL: all in round 0).  The launch runs round 0's instances,
 * then, after a barrier over all its CTAs, round 1's on the same CTAs, and so
 * on; only each round's groups must fit the GPU at once, so a few large
 * instances can take many CTAs in one round and many small ones the next.
 * With ctas == NULL the CTAs of each round are split in proportion to work. */
int fewha_batch_create_rounds(void *const *handles, int n, const int *ctas, const int *rounds, void **batch_out);
/* Same, with the WFS tile of each instance fixed: tiles[2i], tiles[2i+1] =
 * tile rows and columns in pupil nodes (4..64 each, within the shared
 * memory of a CTA; FEWHA_ERR_ARG otherwise), or 0, 0 for the choice of
 * fewha_batch_create for the instance's CTA count.  tiles may be NULL. */
int fewha_batch_create_ex(void *const *handles, int n, const int *ctas, const int *rounds, const int *tiles,
                          void **batch_out);
/* CTAs and WFS tiles (2 ints per instance) of a batch. */
int fewha_batch_ctas(const void *batch, int *ctas_out);
int fewha_batch_tiles(const void *batch, int *tiles_out);
int fewha_batch_solve(void *batch, const void *const *slopes, void *const *c, const fewha_state *states,
                      const fewha_solve_opts *opts, fewha_stats *stats_dev, cudaStream_t stream);
void fewha_batch_destroy(void *batch);

/* Fixed-buffer form for CUDA-graph capture.  fewha_batch_bind writes (and
 * synchronously uploads) the argument table of one batched time step over
 * fixed buffers, with the same arguments and checks as fewha_batch_solve;
 * fewha_batch_launch then runs that time step on `stream` with no host work
 * and no host-to-device copy (two kernel launches: flag reset and the
 * cooperative solve), so it can be captured once into a CUDA graph and
 * replayed every frame after the caller has written the new slopes into the
 * bound slope buffers.  FEWHA_ERR_ARG if nothing is bound. */
int fewha_batch_bind(void *batch, const void *const *slopes, void *const *c, const fewha_state *states,
                     const fewha_solve_opts *opts, fewha_stats *stats_dev);
int fewha_batch_launch(void *batch, cudaStream_t stream);

/* --- Learned warm start (not in the paper) ----------------------------------
 * A small convolutional network over the last frames' layer coefficients
 * predicts the next time step's warm-start increment and deflation
 * directions; PCG stays the solver.  These calls are its building blocks: the
 * network's forward and backward passes, its loss and optimizer, and the
 * deflated warm start that combines the predicted directions with the new
 * data.  FP32 device tensors addressed as base + b*bs + c*cs + y*W + x (batch
 * and channel strides in elements, so that the layers of one grid size form a
 * batch and a channel may be a whole coefficient vector; strides may be
 * negative).  All calls are asynchronous on `s` and return FEWHA_ERR_ARG for
 * NULL pointers or sizes below 1, FEWHA_ERR_CUDA if a launch fails.
 *
 * fewha_conv3x3_fwd: out[b][co] = act(bias[co] + sum_ci w[co][ci] (*) in[b][ci]),
 *   3x3 cross-correlation with zero padding; act = ReLU if relu != 0; w is
 *   Cout x Cin x 3 x 3 (row-major), bias may be NULL.
 * fewha_conv3x3_bwd_data: gin = adjoint of that convolution (no bias, no act)
 *   applied to gout.
 * fewha_conv3x3_bwd_weight: gw (Cout x Cin x 9) and gb (Cout) of
 *   sum_b,co,y,x gout * out; written, or added when accumulate != 0;
 *   workspace: fewha_conv3x3_wgrad_workspace(...) floats; deterministic.
 * fewha_relu_bwd: g[i] = 0 where act[i] <= 0 (act = the ReLU output).
 * fewha_mse_grad: grad = 2 (pred - target) / n; loss_part512[512] partial sums
 *   of (pred - target)^2 (the loss is their sum / n).
 * fewha_adam_step: Adam (Kingma & Ba) with bias correction; step = 1, 2, ...
 * fewha_scale: y = x sqrt(s) (mode 0), x / sqrt(s) (mode 1), y += x / sqrt(s)
 *   (mode 2), elementwise; s > 0 (with s = alpha D this whitens coefficients
 *   by the prior).
 * fewha_learned_targets: targets5 (5 x n) from two consecutive solutions:
 *   t0 = (c_next - c_cur) sqrt(scale), t_k = t0 on coefficients with
 *   group[i] == k and 0 elsewhere (k = 1..4).
 * fewha_deflate_warm_start: Galerkin correction of the warm start over nd
 *   directions D (nd x n, leading dimension ldd) with Q = M D (ldq):
 *   r0 = (b - b_prev) + r_prev (the warm restart of Algorithm 3),
 *   w = (D^T Q)^{-1} D^T r0 in FP64 with a Cholesky factorisation that drops
 *   directions whose pivot is below 1e-10 of their diagonal.  Taken only when
 *   ||r0 - Q w|| < ||r0||; then c += D w and r_prev <- r0 - Q w; otherwise c
 *   is left as it is and r_prev <- r0 (the plain warm start).  Either way
 *   b_prev <- b: this time step's right-hand side is folded into the state,
 *   and the fewha_solve that follows is called with rhs_in_state = 1.
 *   r0_work: n floats; work: FEWHA_DEFLATE_WORK_DOUBLES; info:
 *   FEWHA_DEFLATE_INFO_DOUBLES, info[0] taken (0/1), [1] ||r0 - Q w||,
 *   [2] ||r0||, [3] directions kept, [4..4+nd) w.  1 <= nd <= FEWHA_MAX_DEFLATE. */
#define FEWHA_MAX_DEFLATE 6
#define FEWHA_DEFLATE_WORK_DOUBLES 4096
#define FEWHA_DEFLATE_INFO_DOUBLES 16
int fewha_conv3x3_fwd(const float *in, long in_bs, long in_cs, int Cin, const float *w, const float *bias,
                      float *out, long out_bs, long out_cs, int Cout, int B, int H, int W, int relu, cudaStream_t s);
/* fewha_conv3x3_fwd_tc: the same forward convolution on the tensor cores
 * (tcgen05 implicit GEMM: 128 output pixels per CTA x all output channels,
 * K = 9 Cin): operands rounded to bfloat16, products accumulated in FP32,
 * then bias and ReLU in FP32.  Cin, Cout <= 32.  status_dev (device int, may
 * be NULL) receives FEWHA_ERR_TIMEOUT if a CTA's wait for its tensor-core
 * work ran out (it then frees its tensor memory and leaves its outputs
 * unwritten); it is not cleared by the call.  For inference; training keeps
 * the FP32 kernels. */
int fewha_conv3x3_fwd_tc(const float *in, long in_bs, long in_cs, int Cin, const float *w, const float *bias,
                         float *out, long out_bs, long out_cs, int Cout, int B, int H, int W, int relu,
                         int *status_dev, cudaStream_t s);
int fewha_conv3x3_bwd_data(const float *gout, long gout_bs, long gout_cs, int Cout, const float *w, float *gin,
                           long gin_bs, long gin_cs, int Cin, int B, int H, int W, cudaStream_t s);
long fewha_conv3x3_wgrad_workspace(int Cin, int Cout, int B, int H, int W);
int fewha_conv3x3_bwd_weight(const float *in, long in_bs, long in_cs, int Cin, const float *gout, long gout_bs,
                             long gout_cs, int Cout, int B, int H, int W, float *gw, float *gb, int accumulate,
                             float *workspace, cudaStream_t s);
int fewha_relu_bwd(const float *act, float *g, long n, cudaStream_t s);
int fewha_mse_grad(const float *pred, const float *target, float *grad, long n, double *loss_part512, cudaStream_t s);
int fewha_adam_step(float *param, const float *grad, float *m, float *v, long n, float lr, float beta1, float beta2,
                    float eps, int step, cudaStream_t s);
int fewha_scale(const float *x, const float *s_, float *y, long n, int mode, cudaStream_t s);
int fewha_learned_targets(const float *c_next, const float *c_cur, const float *scale, const signed char *group,
                          float *targets5, long n, cudaStream_t s);
int fewha_deflate_warm_start(const float *b, const float *D, long ldd, const float *Q, long ldq, int nd, float *c,
                             float *b_prev, float *r_prev, long n, float *r0_work, double *work, double *info,
                             cudaStream_t s);

/* Time limit of every device-side wait of the persistent solver (grid
 * barriers), in ns; default 1 s.  A wait that runs out records
 * FEWHA_ERR_TIMEOUT in fewha_stats.status and every CTA returns; the context
 * stays usable.  0 makes any wait time out at once (used to test the error
 * path).  The paper has no counterpart. */
int fewha_set_timeout(void *handle, unsigned long long timeout_ns);

/* Phase trace of the persistent solver (profiling aid).  trace_dev: device
 * buffer of capacity x 4 unsigned 64-bit words, owned by the caller, or NULL
 * to switch tracing off.  Each following fewha_solve (persistent launch)
 * zeroes it and records, per grid barrier i: [4i] the longest time one CTA
 * spent in the phase before it [ns] (from its previous barrier), [4i+1] the
 * %globaltimer when the last CTA finished that phase, [4i+2] when CTA 0
 * passed the barrier, [4i+3] the phase tag.  Barriers
 * beyond the capacity are not recorded.  The paper has no counterpart. */
int fewha_set_trace(void *handle, unsigned long long *trace_dev, int capacity);

/* MCAO fitting onto several deformable mirrors (Sec. 5: the 9-layer MCAO
 * case solves the fitting equation with an unpreconditioned CG of 4
 * iterations; the paper's mirrors are 85x85 at 0 m with 0.5 m pitch, 47x47 at
 * 4 km and 53x53 at 12.7 km with 1 m pitch).  The paper names the step but
 * not its operator; this library's reading: the mirror shapes a = (a_1..a_D)
 * minimise sum_t || P^DM_t a - P^L_t W^{-1} c ||^2 over the fitting
 * directions theta_t, where P^L_t projects every layer onto the (n_s+1)^2
 * pupil nodes in direction theta_t (no cone) and sums them and P^DM_t does the
 * same for the mirrors, both bilinear on their grids; mirror d has
 * dm_n[d]^2 actuators with pitch dm_pitch[d] centred on the axis (actuator i
 * at x = (i - (dm_n[d] - 1)/2) dm_pitch[d]) at altitude dm_h[d].
 * fewha_mcao_fit runs `iters` (0..FEWHA_MAX_ITER) CG iterations on the normal
 * equations from the start the caller puts in `a`, and overwrites `a`.
 * a: device vector of fewha_mcao_n_actuators values in the handle's working
 * precision, mirror after mirror, each row-major (row = y).  c: layer
 * coefficients as for fewha_fit.  The mcao object keeps a pointer to the
 * handle (destroy it first) and owns its own tables and work vectors; calls on
 * one object must not overlap.  FEWHA_ERR_GEOMETRY at creation when a
 * projection leaves a layer grid or a mirror. */
#define FEWHA_MAX_DM 4
#define FEWHA_MAX_DIR 16
typedef struct {
    int n_dm;                          /* 1..FEWHA_MAX_DM */
    int dm_n[FEWHA_MAX_DM];            /* actuators per side (>= 2) */
    double dm_pitch[FEWHA_MAX_DM];     /* [m] */
    double dm_h[FEWHA_MAX_DM];         /* altitude [m] */
    int n_dir;                         /* 1..FEWHA_MAX_DIR */
    double dir_x[FEWHA_MAX_DIR];       /* fitting directions [rad] */
    double dir_y[FEWHA_MAX_DIR];
} fewha_mcao_desc;
int fewha_mcao_create(void *handle, const fewha_mcao_desc *desc, void **mcao_out);
long fewha_mcao_n_actuators(const void *mcao);
int fewha_mcao_fit(void *mcao, const void *c, void *a, int iters, cudaStream_t stream);
void fewha_mcao_destroy(void *mcao);

/* y = M x, like fewha_apply_op, but without allocating anything: no
 * cudaMalloc, no cudaFree, no allocating library call, ever.  Meant for
 * callers that cannot allocate device memory at the point where they apply
 * the operator: a hard real-time control loop that must not stall on the
 * allocator (an allocation can synchronise the device), and plug-ins whose
 * host application owns every device allocation.  The handle itself is
 * still created (and its constant tables allocated) once, beforehand, by
 * fewha_create.
 * The intermediate buffers live in one statically reserved device array of
 * FEWHA_NOALLOC_SCRATCH_BYTES per GPU, held until the process exits.  With
 * CUDA's lazy module loading (the default) the array is reserved on a GPU
 * when the first handle is created there: fewha_create looks up the array's
 * device address (cudaGetSymbolAddress) with the handle's device current,
 * which loads the module holding it, so no later call of this entry point
 * loads anything.  Every call looks the address up again on the current
 * device (no cached pointer outlives a device reset); the current device must
 * be the handle's (FEWHA_ERR_ARG otherwise).  Problems whose buffers do not
 * fit are rejected with FEWHA_ERR_SCRATCH (an ELT-size FP64 operator, n =
 * 98304 with 6 sensors of 84 x 84 subapertures, needs about 4.8 MB).
 * All calls share the one array, which keeps the last call's contents: calls
 * that overlap on the GPU (different streams, different handles on the same
 * device) race and must be ordered by the caller.  The paper has no
 * counterpart; this is a deployment aid.
 * x, y: device vectors of length n, 16-byte aligned, not overlapping. */
#define FEWHA_NOALLOC_SCRATCH_BYTES (8u << 20)
int fewha_apply_op_noalloc(void *handle, const void *x, void *y, cudaStream_t stream);

/* Memory-bandwidth probe (measurement aid; the paper has no counterpart):
 * one launch that reads the `bytes` of device buffer `buf` `reps` times over
 * with 16-byte loads from 4 CTAs of 512 threads per SM, bypassing L1.  Timed
 * by the caller (CUDA events on `stream`); a buffer that fits the
 * L2 cache gives the L2 read bandwidth after the first pass, a larger one the
 * DRAM read bandwidth.  bytes: a positive multiple of 16; buf 16-byte
 * aligned; sink: device array of at least 4 x SMs floats (per-CTA sums, so
 * that no load is dropped).  Asynchronous. */
int fewha_read_probe(const void *buf, long bytes, int reps, float *sink, cudaStream_t stream);

/* Text of a status code. */
/* Copies `bytes` (a multiple of 16, both addresses 16-byte aligned, no
 * overlap) from src to dst with a kernel on `stream`; either side may be
 * device, managed or page-locked host memory (the typical use: a time step's
 * solution into the page-locked buffer the host reads, without a copy-engine
 * transfer on the stream).  FEWHA_ERR_ARG for pageable host memory or bad
 * sizes; asynchronous. */
int fewha_store(void *dst, const void *src, long bytes, cudaStream_t stream);

const char *fewha_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* FEWHA_H */
