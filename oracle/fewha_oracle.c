/*
 * FP64 CPU oracle for the augmented FEWHA hot path (Ramlau & Stadler,
 * "An augmented wavelet reconstructor for atmospheric tomography").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it.  It shares no code,
 * header, table or constant generator with the CUDA library, and the library
 * never calls it.
 *
 * Every routine follows one passage of the paper, written out in the paper's
 * notation, with sequential index-order loops and no blocking or fusion:
 *   - Shack-Hartmann operator Gamma and its adjoint          (Sec. 2)
 *   - NGS / LGS geometric propagation P_g and its adjoint   (Sec. 2)
 *   - periodic orthonormal Daubechies DWT W, W^{-1}          (Sec. 3, Eq. fewha)
 *   - normal operator M and right-hand side b                (Sec. 3, Eq. M)
 *   - diagonal prior D, modified Jacobi preconditioner J      (Sec. 3, Sec. 4)
 *   - PCG (Algorithm 1) and augmented PCG (Algorithm 2)      (Sec. 4)
 *   - warm-restart residual of the reconstructor loop        (Algorithm 3)
 *   - pseudo-open-loop slopes, fitting, gain control          (Algorithm 3)
 * Where the paper is silent or garbled the reading is stated beside the code.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_GEOMETRY (-2)
#define ORC_ERR_BREAKDOWN (-5)
#define ORC_ERR_NOT_SPD (-6)

typedef struct {
    /* telescope (Sec. 5.1 parameter table) */
    double D, obstruction;
    int n_sub;
    /* guide stars: direction theta [rad] and sodium height H [m] (H <= 0 means NGS) */
    int n_gs;
    const double *gs_tx, *gs_ty, *gs_H, *gs_w; /* gs_w = 1/sigma_g^2 (C_eta^{-1}) */
    /* layers: height [m], Cn2 fraction, grid size n_l, wavelet levels J_l, scale delta_l */
    int n_layers;
    const double *lay_h, *lay_cn2, *lay_delta;
    const int *lay_n, *lay_J;
    double r0, alpha;
    int n_taps;
    const double *taps;
    /* subapertures across the sensor of each guide star (NULL or 0: n_sub) */
    const int *gs_ns;
} orc_params;

typedef struct {
    orc_params p;
    /* owned copies of the arrays */
    double *gs_tx, *gs_ty, *gs_H, *gs_w;
    double *lay_h, *lay_cn2, *lay_delta, *taps;
    int *lay_n, *lay_J;
    /* derived geometry */
    double ds;         /* subaperture size D/n_s of the main (mirror) grid */
    int *gns;          /* per guide star: subapertures across its sensor */
    double *gds;       /* per guide star: its subaperture size D/n_g */
    long *slope_off;   /* per guide star: offset of its slopes (2 n_g^2 each), n_gs + 1 */
    long *mask_off;    /* per guide star: offset of its mask (n_g^2 each), n_gs + 1 */
    unsigned char *mask; /* valid subapertures, sensor after sensor */
    double *lay_d;     /* layer grid spacing */
    long *lay_off;     /* offset of layer l in the coefficient vector */
    long n;            /* total unknowns */
    double *prior;     /* D diagonal, n */
    double *invJ;      /* J^{-1} diagonal, n */
} orc_ctx;

/* ------------------------------------------------------------------------ */
/* Geometry (Sec. 2, Sec. 3, Fig. grids)                                     */
/* ------------------------------------------------------------------------ */

/* Pupil node (i, j): x = -D/2 + j*ds (first axis), y = -D/2 + i*ds; ds of
 * the main grid (the mirror's actuators) or of guide star g's sensor. */
static double pupil_coord(const orc_ctx *c, int idx) { return -0.5 * c->p.D + idx * c->ds; }
static double pupil_coord_g(const orc_ctx *c, int g, int idx) { return -0.5 * c->p.D + idx * c->gds[g]; }

/* Cone compression factor of guide star g at height h: 1 for an NGS,
 * 1 - h/H for an LGS at height H (Sec. 2, P^LGS). */
static double cone_scale(const orc_ctx *c, int g, double h)
{
    double H = c->p.gs_H[g];
    return (H > 0.0) ? (1.0 - h / H) : 1.0;
}

/* Reading of the layer domain Omega_l (not given in the paper): an n_l x n_l
 * node grid, node k at coordinate (k - n_l/2) * d_l on each axis, with d_l the
 * smallest spacing such that every projected pupil node of every guide star
 * lies at least one cell inside the grid: R_l / d_l = n_l/2 - 2, where R_l is
 * the largest |coordinate| of a projected pupil node. */
static double layer_radius(const orc_ctx *c, int l)
{
    double h = c->p.lay_h[l], R = 0.0;
    for (int g = 0; g < c->p.n_gs; g++) {
        double s = cone_scale(c, g, h);
        double tx = fabs(c->p.gs_tx[g] * h), ty = fabs(c->p.gs_ty[g] * h);
        double r = s * 0.5 * c->p.D + (tx > ty ? tx : ty);
        if (r > R) R = r;
    }
    return R;
}

/* ------------------------------------------------------------------------ */
/* Wavelets (Sec. 3, Eq. fewha): periodic orthonormal DWT                    */
/* ------------------------------------------------------------------------ */

/* One analysis level on a periodic line of length N (N even):
 *   a_k = sum_n h_n x_{(2k+n) mod N},  d_k = sum_n g_n x_{(2k+n) mod N},
 *   g_n = (-1)^n h_{L-1-n};  output [a_0..a_{N/2-1}, d_0..d_{N/2-1}]. */
void orc_dwt1_fwd(int N, int L, const double *h, const double *x, double *out)
{
    int half = N / 2;
    for (int k = 0; k < half; k++) {
        double a = 0.0, d = 0.0;
        for (int t = 0; t < L; t++) {
            double g = ((t & 1) ? -1.0 : 1.0) * h[L - 1 - t];
            double v = x[(2 * k + t) % N];
            a += h[t] * v;
            d += g * v;
        }
        out[k] = a;
        out[half + k] = d;
    }
}

/* Synthesis = exact transpose of the analysis level above. */
void orc_dwt1_inv(int N, int L, const double *h, const double *ad, double *x)
{
    int half = N / 2;
    for (int i = 0; i < N; i++) x[i] = 0.0;
    for (int k = 0; k < half; k++) {
        for (int t = 0; t < L; t++) {
            double g = ((t & 1) ? -1.0 : 1.0) * h[L - 1 - t];
            x[(2 * k + t) % N] += h[t] * ad[k] + g * ad[half + k];
        }
    }
}

/* 2-D Mallat pyramid on an n x n row-major array, J levels fine -> coarse:
 * level t works on the top-left (n>>t) x (n>>t) block, rows then columns. */
void orc_dwt2_fwd(int n, int J, int L, const double *h, const double *in, double *out)
{
    double *line = malloc(sizeof(double) * n), *tmp = malloc(sizeof(double) * n);
    memcpy(out, in, sizeof(double) * n * n);
    for (int t = 0; t < J; t++) {
        int N = n >> t;
        for (int r = 0; r < N; r++) {
            for (int q = 0; q < N; q++) line[q] = out[r * n + q];
            orc_dwt1_fwd(N, L, h, line, tmp);
            for (int q = 0; q < N; q++) out[r * n + q] = tmp[q];
        }
        for (int q = 0; q < N; q++) {
            for (int r = 0; r < N; r++) line[r] = out[r * n + q];
            orc_dwt1_fwd(N, L, h, line, tmp);
            for (int r = 0; r < N; r++) out[r * n + q] = tmp[r];
        }
    }
    free(line);
    free(tmp);
}

/* Inverse pyramid, coarse -> fine, each level the transpose of the forward one
 * (columns then rows). */
void orc_dwt2_inv(int n, int J, int L, const double *h, const double *in, double *out)
{
    double *line = malloc(sizeof(double) * n), *tmp = malloc(sizeof(double) * n);
    memcpy(out, in, sizeof(double) * n * n);
    for (int t = J - 1; t >= 0; t--) {
        int N = n >> t;
        for (int q = 0; q < N; q++) {
            for (int r = 0; r < N; r++) line[r] = out[r * n + q];
            orc_dwt1_inv(N, L, h, line, tmp);
            for (int r = 0; r < N; r++) out[r * n + q] = tmp[r];
        }
        for (int r = 0; r < N; r++) {
            for (int q = 0; q < N; q++) line[q] = out[r * n + q];
            orc_dwt1_inv(N, L, h, line, tmp);
            for (int q = 0; q < N; q++) out[r * n + q] = tmp[q];
        }
    }
    free(line);
    free(tmp);
}

/* Block-diagonal W = diag(delta_l W) (Eq. fewha): W^{-1} = W^T / delta_l. */
static void W_inv(const orc_ctx *c, const double *coef, double *nodal)
{
    for (int l = 0; l < c->p.n_layers; l++) {
        int n = c->lay_n[l];
        long o = c->lay_off[l];
        orc_dwt2_inv(n, c->lay_J[l], c->p.n_taps, c->taps, coef + o, nodal + o);
        for (long i = 0; i < (long)n * n; i++) nodal[o + i] /= c->lay_delta[l];
    }
}

/* W^{-T} = W / delta_l. */
static void W_invT(const orc_ctx *c, const double *nodal, double *coef)
{
    for (int l = 0; l < c->p.n_layers; l++) {
        int n = c->lay_n[l];
        long o = c->lay_off[l];
        orc_dwt2_fwd(n, c->lay_J[l], c->p.n_taps, c->taps, nodal + o, coef + o);
        for (long i = 0; i < (long)n * n; i++) coef[o + i] /= c->lay_delta[l];
    }
}

/* ------------------------------------------------------------------------ */
/* Geometric propagation (Sec. 2): phi_g(x) = sum_l phi_l((1-h_l/H)x + theta h_l) */
/* ------------------------------------------------------------------------ */

/* Bilinear position on layer l of the pupil coordinate pair (x, y) for g:
 * returns the lower node index and fractional weight on each axis. */
static int layer_position(const orc_ctx *c, int g, int l, double x, double y,
                          int *kx, int *ky, double *wx, double *wy)
{
    double h = c->p.lay_h[l], s = cone_scale(c, g, h), d = c->lay_d[l];
    int n = c->lay_n[l];
    double px = s * x + c->p.gs_tx[g] * h;
    double py = s * y + c->p.gs_ty[g] * h;
    double fx = px / d + 0.5 * n, fy = py / d + 0.5 * n;
    *kx = (int)floor(fx);
    *ky = (int)floor(fy);
    *wx = fx - *kx;
    *wy = fy - *ky;
    if (*kx < 0 || *ky < 0 || *kx + 1 > n - 1 || *ky + 1 > n - 1) return ORC_ERR_GEOMETRY;
    return ORC_OK;
}

/* P_g: layers (nodal) -> wavefront on the (n_g+1)^2 pupil nodes of g's sensor. */
void orc_prop_fwd(const orc_ctx *c, int g, const double *nodal, double *wf)
{
    int m = c->gns[g] + 1;
    for (int i = 0; i < m; i++) {
        for (int j = 0; j < m; j++) {
            double x = pupil_coord_g(c, g, j), y = pupil_coord_g(c, g, i), v = 0.0;
            for (int l = 0; l < c->p.n_layers; l++) {
                int kx, ky, n = c->lay_n[l];
                double wx, wy;
                layer_position(c, g, l, x, y, &kx, &ky, &wx, &wy);
                const double *L = nodal + c->lay_off[l];
                v += (1 - wy) * ((1 - wx) * L[ky * n + kx] + wx * L[ky * n + kx + 1]) +
                     wy * ((1 - wx) * L[(ky + 1) * n + kx] + wx * L[(ky + 1) * n + kx + 1]);
            }
            wf[i * m + j] = v;
        }
    }
}

/* P_g^T: scatter form of the exact transpose (accumulates into nodal). */
void orc_prop_adj(const orc_ctx *c, int g, const double *wf, double *nodal)
{
    int m = c->gns[g] + 1;
    for (int i = 0; i < m; i++) {
        for (int j = 0; j < m; j++) {
            double x = pupil_coord_g(c, g, j), y = pupil_coord_g(c, g, i), v = wf[i * m + j];
            for (int l = 0; l < c->p.n_layers; l++) {
                int kx, ky, n = c->lay_n[l];
                double wx, wy;
                layer_position(c, g, l, x, y, &kx, &ky, &wx, &wy);
                double *L = nodal + c->lay_off[l];
                L[ky * n + kx] += (1 - wy) * (1 - wx) * v;
                L[ky * n + kx + 1] += (1 - wy) * wx * v;
                L[(ky + 1) * n + kx] += wy * (1 - wx) * v;
                L[(ky + 1) * n + kx + 1] += wy * wx * v;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Shack-Hartmann operator Gamma (Sec. 2)                                   */
/* ------------------------------------------------------------------------ */

/* s^x_ij = [(phi_{i,j+1}-phi_{i,j}) + (phi_{i+1,j+1}-phi_{i+1,j})]/2
 * s^y_ij = [(phi_{i+1,j}-phi_{i,j}) + (phi_{i+1,j+1}-phi_{i,j+1})]/2
 * (the y formula as printed has a diagonal second difference; the reading is
 * the x/y-symmetric form).  Output [x block | y block], n_s^2 each. */
void orc_gamma_fwd(int ns, const double *wf, double *s)
{
    int m = ns + 1;
    for (int i = 0; i < ns; i++) {
        for (int j = 0; j < ns; j++) {
            double p00 = wf[i * m + j], p01 = wf[i * m + j + 1];
            double p10 = wf[(i + 1) * m + j], p11 = wf[(i + 1) * m + j + 1];
            s[i * ns + j] = 0.5 * ((p01 - p00) + (p11 - p10));
            s[ns * ns + i * ns + j] = 0.5 * ((p10 - p00) + (p11 - p01));
        }
    }
}

/* Gamma^T in scatter form (accumulates into wf). */
void orc_gamma_adj(int ns, const double *s, double *wf)
{
    int m = ns + 1;
    for (int i = 0; i < ns; i++) {
        for (int j = 0; j < ns; j++) {
            double sx = 0.5 * s[i * ns + j], sy = 0.5 * s[ns * ns + i * ns + j];
            wf[i * m + j] += -sx - sy;
            wf[i * m + j + 1] += sx - sy;
            wf[(i + 1) * m + j] += -sx + sy;
            wf[(i + 1) * m + j + 1] += sx + sy;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Tomography operator A = (Gamma_g P_g)_g, noise weight, M and b (Sec. 3)   */
/* ------------------------------------------------------------------------ */

long orc_n_unknowns(const orc_ctx *c) { return c->n; }
long orc_n_slopes(const orc_ctx *c) { return c->slope_off[c->p.n_gs]; }
long orc_slope_offset(const orc_ctx *c, int g) { return c->slope_off[g]; }
int orc_sensor_ns(const orc_ctx *c, int g) { return c->gns[g]; }
double orc_layer_spacing(const orc_ctx *c, int l) { return c->lay_d[l]; }
const unsigned char *orc_mask(const orc_ctx *c) { return c->mask; }

/* s = A phi (all guide stars, all subapertures, no weighting). */
void orc_apply_A(const orc_ctx *c, const double *nodal, double *s)
{
    for (int g = 0; g < c->p.n_gs; g++) {
        int ns = c->gns[g], m = ns + 1;
        double *wf = malloc(sizeof(double) * m * m);
        orc_prop_fwd(c, g, nodal, wf);
        orc_gamma_fwd(ns, wf, s + c->slope_off[g]);
        free(wf);
    }
}

/* phi = A^T s (overwrites phi). */
void orc_apply_AT(const orc_ctx *c, const double *s, double *nodal)
{
    memset(nodal, 0, sizeof(double) * c->n);
    for (int g = 0; g < c->p.n_gs; g++) {
        int ns = c->gns[g], m = ns + 1;
        double *wf = calloc((size_t)m * m, sizeof(double));
        orc_gamma_adj(ns, s + c->slope_off[g], wf);
        orc_prop_adj(c, g, wf, nodal);
        free(wf);
    }
}

/* C_eta^{-1}: diagonal, 1/sigma_g^2 on valid subapertures and 0 elsewhere
 * (reading of the noise covariance; the paper gives no form). */
void orc_apply_Cinv(const orc_ctx *c, double *s)
{
    for (int g = 0; g < c->p.n_gs; g++) {
        int ns = c->gns[g];
        double w = c->p.gs_w[g];
        for (int a = 0; a < 2; a++)
            for (int i = 0; i < ns * ns; i++) {
                long k = c->slope_off[g] + (long)a * ns * ns + i;
                s[k] = c->mask[c->mask_off[g] + i] ? w * s[k] : 0.0;
            }
    }
}

/* y = M x = W^{-T} A^T C_eta^{-1} A W^{-1} x + alpha D x   (Eq. M) */
void orc_apply_op(const orc_ctx *c, const double *x, double *y)
{
    long n = c->n, ns2 = orc_n_slopes(c);
    double *v = malloc(sizeof(double) * n), *u = malloc(sizeof(double) * n);
    double *s = malloc(sizeof(double) * ns2);
    W_inv(c, x, v);
    orc_apply_A(c, v, s);
    orc_apply_Cinv(c, s);
    orc_apply_AT(c, s, u);
    W_invT(c, u, y);
    for (long i = 0; i < n; i++) y[i] += c->p.alpha * c->prior[i] * x[i];
    free(v);
    free(u);
    free(s);
}

/* b = W^{-T} A^T C_eta^{-1} s   (Sec. 3, right-hand side; Algorithm 3 RHS step) */
void orc_rhs(const orc_ctx *c, const double *s_in, double *b)
{
    long n = c->n, ns2 = orc_n_slopes(c);
    double *s = malloc(sizeof(double) * ns2), *u = malloc(sizeof(double) * n);
    memcpy(s, s_in, sizeof(double) * ns2);
    orc_apply_Cinv(c, s);
    orc_apply_AT(c, s, u);
    W_invT(c, u, b);
    free(s);
    free(u);
}

/* ------------------------------------------------------------------------ */
/* Mirror side of the reconstructor loop (Algorithm 3)                       */
/* Reading: one deformable mirror conjugated to the ground whose actuators   */
/* sit on the (n_s+1)^2 pupil nodes (the subaperture corners); the phase it  */
/* adds at a pupil node is its actuator value there, the same for every      */
/* guide star (no cone, no shift at height 0).                               */
/* ------------------------------------------------------------------------ */

/* Fitting step a~ = F W^{-1} c: the on-axis projection (direction 0, no cone)
 * of every layer onto the actuators, bilinear on each layer grid.  Returns
 * ORC_ERR_GEOMETRY if an actuator projects outside a layer grid. */
int orc_fit(const orc_ctx *c, const double *coef, double *a)
{
    int m = c->p.n_sub + 1;
    double *nodal = malloc(sizeof(double) * c->n);
    W_inv(c, coef, nodal);
    int st = ORC_OK;
    for (int i = 0; i < m && st == ORC_OK; i++) {
        for (int j = 0; j < m; j++) {
            double x = pupil_coord(c, j), y = pupil_coord(c, i), v = 0.0;
            for (int l = 0; l < c->p.n_layers; l++) {
                int n = c->lay_n[l];
                double d = c->lay_d[l];
                double fx = x / d + 0.5 * n, fy = y / d + 0.5 * n;
                int kx = (int)floor(fx), ky = (int)floor(fy);
                double wx = fx - kx, wy = fy - ky;
                if (kx < 0 || ky < 0 || kx + 1 > n - 1 || ky + 1 > n - 1) {
                    st = ORC_ERR_GEOMETRY;
                    break;
                }
                const double *L = nodal + c->lay_off[l];
                v += (1 - wy) * ((1 - wx) * L[ky * n + kx] + wx * L[ky * n + kx + 1]) +
                     wy * ((1 - wx) * L[(ky + 1) * n + kx] + wx * L[(ky + 1) * n + kx + 1]);
            }
            a[i * m + j] = v;
        }
    }
    free(nodal);
    return st;
}

/* Pseudo-open-loop measurements (closed loop): s_out = s + Gamma a for every
 * guide star, a the mirror shape applied two steps earlier.  The mirror's
 * actuators sit on the main pupil grid, so every sensor must have the main
 * n_sub (ORC_ERR_GEOMETRY otherwise). */
int orc_pol_slopes(const orc_ctx *c, const double *s, const double *a, double *s_out)
{
    int ns = c->p.n_sub;
    for (int g = 0; g < c->p.n_gs; g++)
        if (c->gns[g] != ns) return ORC_ERR_GEOMETRY;
    long per = 2L * ns * ns;
    double *ga = malloc(sizeof(double) * per);
    orc_gamma_fwd(ns, a, ga);
    for (int g = 0; g < c->p.n_gs; g++)
        for (long e = 0; e < per; e++) s_out[g * per + e] = s[g * per + e] + ga[e];
    free(ga);
    return ORC_OK;
}

/* Gain control: closed loop a_next = a_i + gain (a~ - a_{i-1}); open loop
 * a_next = (1 - gain) a_i + gain a~. */
void orc_control(long na, int closed, double gain, const double *a_im1, const double *a_i,
                 const double *a_fit, double *a_next)
{
    for (long e = 0; e < na; e++)
        a_next[e] = closed ? a_i[e] + gain * (a_fit[e] - a_im1[e]) : (1.0 - gain) * a_i[e] + gain * a_fit[e];
}

/* ------------------------------------------------------------------------ */
/* Prior D and preconditioner J (Sec. 3, Sec. 4)                            */
/* ------------------------------------------------------------------------ */

/* Band of coefficient (r, q) of an n x n Mallat layout with J levels:
 * s = 0 for the coarsest approximation block, s = 1..J for the detail bands
 * from coarse to fine; quadrant 0 approximation, 1 (low y, high x),
 * 2 (high y, low x), 3 (high-high). */
void orc_band_of(int n, int J, int r, int q, int *s, int *quad)
{
    int a = n >> J;
    if (r < a && q < a) {
        *s = 0;
        *quad = 0;
        return;
    }
    for (int lev = 1; lev <= J; lev++) {
        int half = a << (lev - 1); /* band size at coarse-to-fine level lev */
        if (r < 2 * half && q < 2 * half) {
            *s = lev;
            *quad = (r < half) ? 1 : ((q < half) ? 2 : 3);
            return;
        }
    }
    *s = -1;
    *quad = -1;
}

/* Reading of D (the paper says only "diagonal approximation of C_phi^{-1} in
 * the frequency domain"): for a Kolmogorov layer with Fried parameter
 * r0_l = r0 * cn2_l^{-3/5}, the variance of an orthonormal detail coefficient
 * at the finest level is taken as 0.5 * 6.88 (d_l / r0_l)^{5/3} and grows by
 * 2^{11/3} per coarser level, so
 *   D = kappa_l 2^{(11/3) s},  kappa_l = 2^{-(11/3) J_l} / (0.5 * 6.88 (d_l/r0_l)^{5/3}),
 * with s = 0 for the approximation block. */
static void build_prior(orc_ctx *c)
{
    for (int l = 0; l < c->p.n_layers; l++) {
        int n = c->lay_n[l], J = c->lay_J[l];
        double r0l = c->p.r0 * pow(c->lay_cn2[l], -3.0 / 5.0);
        double kappa = pow(2.0, -(11.0 / 3.0) * J) / (0.5 * 6.88 * pow(c->lay_d[l] / r0l, 5.0 / 3.0));
        for (int r = 0; r < n; r++)
            for (int q = 0; q < n; q++) {
                int s, quad;
                orc_band_of(n, J, r, q, &s, &quad);
                c->prior[c->lay_off[l] + (long)r * n + q] = kappa * pow(2.0, (11.0 / 3.0) * s);
            }
    }
}

/* Data-term diagonal entry e_i^T W^{-T} A^T C A W^{-1} e_i = ||C^{1/2} A W^{-1} e_i||^2. */
double orc_data_diag(const orc_ctx *c, long i)
{
    long n = c->n, ns2 = orc_n_slopes(c);
    double *e = calloc(n, sizeof(double)), *v = malloc(sizeof(double) * n);
    double *s = malloc(sizeof(double) * ns2);
    e[i] = 1.0;
    W_inv(c, e, v);
    orc_apply_A(c, v, s);
    double acc = 0.0;
    for (int g = 0; g < c->p.n_gs; g++) {
        int ns = c->gns[g];
        for (int a = 0; a < 2; a++)
            for (int k = 0; k < ns * ns; k++) {
                double val = s[c->slope_off[g] + (long)a * ns * ns + k];
                if (c->mask[c->mask_off[g] + k]) acc += c->p.gs_w[g] * val * val;
            }
    }
    free(e);
    free(v);
    free(s);
    return acc;
}

/* Reading of the modified Jacobi preconditioner (Sec. 4, "different weighting
 * of low and high frequencies", weights not given):
 *   J_ii = alpha D_ii + t_{l,s,quad},
 * t = mean of the data-term diagonal over sample coefficients of the same
 * layer and band; the samples sit at offsets {floor(nb/4), floor(3nb/4)} on
 * each axis of the nb x nb band (duplicates dropped). */
static void build_precond(orc_ctx *c)
{
    for (int l = 0; l < c->p.n_layers; l++) {
        int n = c->lay_n[l], J = c->lay_J[l];
        double t[64][4];
        for (int s = 0; s <= J; s++) {
            int nb = (n >> J) << (s > 0 ? s - 1 : 0);
            for (int quad = (s == 0 ? 0 : 1); quad <= (s == 0 ? 0 : 3); quad++) {
                int r0 = (quad == 2 || quad == 3) ? nb : 0;
                int q0 = (quad == 1 || quad == 3) ? nb : 0;
                int offs[2] = {nb / 4, (3 * nb) / 4}, no = (offs[0] == offs[1]) ? 1 : 2;
                double acc = 0.0;
                int cnt = 0;
                for (int a = 0; a < no; a++)
                    for (int b = 0; b < no; b++) {
                        long idx = c->lay_off[l] + (long)(r0 + offs[a]) * n + (q0 + offs[b]);
                        acc += orc_data_diag(c, idx);
                        cnt++;
                    }
                t[s][quad] = acc / cnt;
            }
        }
        for (int r = 0; r < n; r++)
            for (int q = 0; q < n; q++) {
                int s, quad;
                orc_band_of(n, J, r, q, &s, &quad);
                long i = c->lay_off[l] + (long)r * n + q;
                c->invJ[i] = 1.0 / (c->p.alpha * c->prior[i] + t[s][quad]);
            }
    }
}

const double *orc_prior(const orc_ctx *c) { return c->prior; }
const double *orc_invJ(const orc_ctx *c) { return c->invJ; }

/* ------------------------------------------------------------------------ */
/* Construction                                                               */
/* ------------------------------------------------------------------------ */

static double *dupd(const double *a, int n)
{
    double *r = malloc(sizeof(double) * (n > 0 ? n : 1));
    if (n > 0) memcpy(r, a, sizeof(double) * n);
    return r;
}

void orc_destroy(orc_ctx *c);

/* with_precond = 0 leaves J^{-1} = 1 (identity) and skips the sampling. */
int orc_create(const orc_params *p, int with_precond, orc_ctx **out)
{
    *out = NULL;
    if (p->n_sub < 1 || p->n_gs < 1 || p->n_layers < 1 || p->n_taps < 2 || p->D <= 0) return ORC_ERR_ARG;
    orc_ctx *c = calloc(1, sizeof(orc_ctx));
    c->p = *p;
    c->gs_tx = dupd(p->gs_tx, p->n_gs);
    c->gs_ty = dupd(p->gs_ty, p->n_gs);
    c->gs_H = dupd(p->gs_H, p->n_gs);
    c->gs_w = dupd(p->gs_w, p->n_gs);
    c->lay_h = dupd(p->lay_h, p->n_layers);
    c->lay_cn2 = dupd(p->lay_cn2, p->n_layers);
    c->lay_delta = dupd(p->lay_delta, p->n_layers);
    c->taps = dupd(p->taps, p->n_taps);
    c->lay_n = malloc(sizeof(int) * p->n_layers);
    c->lay_J = malloc(sizeof(int) * p->n_layers);
    memcpy(c->lay_n, p->lay_n, sizeof(int) * p->n_layers);
    memcpy(c->lay_J, p->lay_J, sizeof(int) * p->n_layers);
    c->p.gs_tx = c->gs_tx;
    c->p.gs_ty = c->gs_ty;
    c->p.gs_H = c->gs_H;
    c->p.gs_w = c->gs_w;
    c->p.lay_h = c->lay_h;
    c->p.lay_cn2 = c->lay_cn2;
    c->p.lay_delta = c->lay_delta;
    c->p.taps = c->taps;
    c->p.lay_n = c->lay_n;
    c->p.lay_J = c->lay_J;

    c->ds = p->D / p->n_sub;
    /* sensors: guide star g has an n_g x n_g Shack-Hartmann sensor over the
     * pupil; a subaperture is lit iff its centre radius is within
     * [obstruction D/2, D/2], except that the single subaperture of a 1x1
     * sensor sees the whole pupil and is always lit (reading) */
    int G = p->n_gs;
    c->gns = malloc(sizeof(int) * G);
    c->gds = malloc(sizeof(double) * G);
    c->slope_off = malloc(sizeof(long) * (G + 1));
    c->mask_off = malloc(sizeof(long) * (G + 1));
    c->slope_off[0] = c->mask_off[0] = 0;
    for (int g = 0; g < G; g++) {
        int ns = (p->gs_ns && p->gs_ns[g] > 0) ? p->gs_ns[g] : p->n_sub;
        c->gns[g] = ns;
        c->gds[g] = p->D / ns;
        c->slope_off[g + 1] = c->slope_off[g] + 2L * ns * ns;
        c->mask_off[g + 1] = c->mask_off[g] + (long)ns * ns;
    }
    c->p.gs_ns = NULL;
    c->mask = malloc(c->mask_off[G] > 0 ? c->mask_off[G] : 1);
    double rin = 0.5 * p->obstruction * p->D, rout = 0.5 * p->D;
    for (int g = 0; g < G; g++) {
        int ns = c->gns[g];
        for (int i = 0; i < ns; i++)
            for (int j = 0; j < ns; j++) {
                double cx = -0.5 * p->D + (j + 0.5) * c->gds[g], cy = -0.5 * p->D + (i + 0.5) * c->gds[g];
                double r = sqrt(cx * cx + cy * cy);
                c->mask[c->mask_off[g] + i * ns + j] = (ns == 1 || (r >= rin && r <= rout)) ? 1 : 0;
            }
    }

    c->lay_d = malloc(sizeof(double) * p->n_layers);
    c->lay_off = malloc(sizeof(long) * (p->n_layers + 1));
    c->n = 0;
    for (int l = 0; l < p->n_layers; l++) {
        int n = p->lay_n[l], J = p->lay_J[l];
        if (n < 8 || (n & (n - 1)) || J < 1 || (n >> J) < 1 || p->lay_cn2[l] <= 0 || p->lay_delta[l] == 0) {
            orc_destroy(c);
            return ORC_ERR_GEOMETRY;
        }
        for (int g = 0; g < p->n_gs; g++)
            if (p->gs_H[g] > 0 && p->lay_h[l] >= p->gs_H[g]) {
                orc_destroy(c);
                return ORC_ERR_GEOMETRY;
            }
        c->lay_d[l] = layer_radius(c, l) / (0.5 * n - 2.0);
        c->lay_off[l] = c->n;
        c->n += (long)n * n;
    }
    c->lay_off[p->n_layers] = c->n;
    c->prior = malloc(sizeof(double) * c->n);
    c->invJ = malloc(sizeof(double) * c->n);
    build_prior(c);
    if (with_precond)
        build_precond(c);
    else
        for (long i = 0; i < c->n; i++) c->invJ[i] = 1.0;
    *out = c;
    return ORC_OK;
}

/* Replace J^{-1} (used by tests that pin the solver with exact Jacobi). */
void orc_set_invJ(orc_ctx *c, const double *invJ) { memcpy(c->invJ, invJ, sizeof(double) * c->n); }

void orc_destroy(orc_ctx *c)
{
    if (!c) return;
    free(c->gs_tx); free(c->gs_ty); free(c->gs_H); free(c->gs_w);
    free(c->lay_h); free(c->lay_cn2); free(c->lay_delta); free(c->taps);
    free(c->lay_n); free(c->lay_J); free(c->mask); free(c->lay_d); free(c->lay_off);
    free(c->gns); free(c->gds); free(c->slope_off); free(c->mask_off);
    free(c->prior); free(c->invJ);
    free(c);
}

/* ------------------------------------------------------------------------ */
/* PCG (Algorithm 1) and augmented PCG (Algorithm 2)                         */
/* ------------------------------------------------------------------------ */

static double dot(long n, const double *a, const double *b)
{
    double s = 0.0;
    for (long i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* Cholesky of a k x k SPD matrix (row-major, lower factor in place). */
static int chol(int k, double *A)
{
    for (int j = 0; j < k; j++) {
        double s = A[j * k + j];
        for (int t = 0; t < j; t++) s -= A[j * k + t] * A[j * k + t];
        if (!(s > 0.0)) return ORC_ERR_NOT_SPD;
        A[j * k + j] = sqrt(s);
        for (int i = j + 1; i < k; i++) {
            double v = A[i * k + j];
            for (int t = 0; t < j; t++) v -= A[i * k + t] * A[j * k + t];
            A[i * k + j] = v / A[j * k + j];
        }
    }
    return ORC_OK;
}

static void chol_solve(int k, const double *Lf, const double *rhs, double *x)
{
    for (int i = 0; i < k; i++) {
        double v = rhs[i];
        for (int t = 0; t < i; t++) v -= Lf[i * k + t] * x[t];
        x[i] = v / Lf[i * k + i];
    }
    for (int i = k - 1; i >= 0; i--) {
        double v = x[i];
        for (int t = i + 1; t < k; t++) v -= Lf[t * k + i] * x[t];
        x[i] = v / Lf[i * k + i];
    }
}

typedef struct {
    int max_iter;      /* iterations k = 0..max_iter-1 (Algorithm 1 loop, reading) */
    double rtol;       /* > 0: stop when ||r|| <= rtol ||b|| */
    int augmented;     /* 0: Algorithm 1, 1: Algorithm 2 */
    int init_mode;     /* 0: Gram form sigma = G^{-1} P^T r, 1: the paper's sequential sigma_j */
    int loop_mode;     /* 0: project z against the newest recycled direction p_m (paper), 1: against all */
    int true_residual_init; /* 1: r0 = b - M c instead of (b - b_prev) + r_prev */
    int true_res_every;     /* N > 0: after every N-th iteration r <- b - M c (residual replacement) */
} orc_opts;

typedef struct {
    int iterations;
    double rel_res;   /* ||r|| / ||b|| (recurrence residual) */
    double bnorm;
    int status;
} orc_stats;

/* Projection of v against the basis in Gram form: tau = Gs^{-1} (X^T v). */
static int gram_coeffs(long n, int k, const double *P, const double *Q, const double *X,
                       const double *v, double *tau)
{
    double G[64 * 64], rhs[64];
    for (int i = 0; i < k; i++)
        for (int j = 0; j < k; j++) G[i * k + j] = dot(n, P + i * n, Q + j * n);
    for (int i = 0; i < k; i++)
        for (int j = 0; j < i; j++) {
            double s = 0.5 * (G[i * k + j] + G[j * k + i]);
            G[i * k + j] = G[j * k + i] = s;
        }
    for (int i = 0; i < k; i++) rhs[i] = dot(n, X + i * n, v);
    int st = chol(k, G);
    if (st) return st;
    chol_solve(k, G, rhs, tau);
    return ORC_OK;
}

/*
 * One reconstructor time step (Algorithm 3 RHS and residual steps, then
 * Algorithm 1 or 2):
 *   b = W^{-T} A^T C_eta^{-1} s;  r0 = (b - b_prev) + r_prev;  b_prev <- b
 *   [c, r, P, Q, pq] <- (aug)PCG(c, r0, J^{-1}, P, Q, pq)
 * Basis P, Q: kcap x n row blocks, oldest first, *k_valid of them in use;
 * pq[j] = (p_j, q_j).  After the solve the basis holds the last
 * min(iterations, kcap) directions of this solve (unchanged if none ran).
 * hist (optional): per iteration k the vectors r_k, z_k, p_k, q_k
 * (4 x (max_iter+1) x n doubles) for invariant tests.
 */
int orc_solve(const orc_ctx *cx, const double *s, double *c, double *b_prev, double *r_prev,
              double *P, double *Q, double *pq, int kcap, int *k_valid,
              const orc_opts *o, orc_stats *st, double *hist)
{
    long n = cx->n;
    int kv = *k_valid, status = ORC_OK;
    double *b = malloc(sizeof(double) * n), *r = malloc(sizeof(double) * n);
    double *z = malloc(sizeof(double) * n), *p = malloc(sizeof(double) * n);
    double *q = malloc(sizeof(double) * n), *tmp = malloc(sizeof(double) * n);
    int cap_iter = o->max_iter > 0 ? o->max_iter : 1;
    double *newP = malloc(sizeof(double) * n * cap_iter), *newQ = malloc(sizeof(double) * n * cap_iter);
    double *newpq = malloc(sizeof(double) * cap_iter);
    double tau[64];

    orc_rhs(cx, s, b);
    if (o->true_residual_init) {
        orc_apply_op(cx, c, tmp);
        for (long i = 0; i < n; i++) r[i] = b[i] - tmp[i];
    } else {
        for (long i = 0; i < n; i++) r[i] = (b[i] - b_prev[i]) + r_prev[i];
    }
    memcpy(b_prev, b, sizeof(double) * n);
    double bnorm = sqrt(dot(n, b, b));
    int aug = o->augmented && kv > 0;

    /* Algorithm 2, initial-guess projection: P^T r0 = 0 afterwards. */
    if (aug) {
        if (o->init_mode == 0) {
            status = gram_coeffs(n, kv, P, Q, P, r, tau);
            if (status) goto done;
            for (int j = 0; j < kv; j++)
                for (long i = 0; i < n; i++) {
                    c[i] += tau[j] * P[j * n + i];
                    r[i] -= tau[j] * Q[j * n + i];
                }
        } else {
            for (int j = 0; j < kv; j++) {
                double sig = dot(n, r, P + j * n) / pq[j];
                for (long i = 0; i < n; i++) {
                    c[i] += sig * P[j * n + i];
                    r[i] -= sig * Q[j * n + i];
                }
            }
        }
    }
    for (long i = 0; i < n; i++) z[i] = cx->invJ[i] * r[i];
    /* Algorithm 2, initial direction: z0 <- z0 - [(z0,q_j)/(p_j,q_j)] p_j (the
     * printed line omits the vector p_j; the reading restores it). */
    if (aug) {
        if (o->init_mode == 0) {
            status = gram_coeffs(n, kv, P, Q, Q, z, tau);
            if (status) goto done;
            for (int j = 0; j < kv; j++)
                for (long i = 0; i < n; i++) z[i] -= tau[j] * P[j * n + i];
        } else {
            for (int j = 0; j < kv; j++) {
                double mu = dot(n, z, Q + j * n) / pq[j];
                for (long i = 0; i < n; i++) z[i] -= mu * P[j * n + i];
            }
        }
    }
    /* p_0 = z_0 (Algorithm 1 prints p_0 = r_0; preconditioned CG needs z_0). */
    memcpy(p, z, sizeof(double) * n);
    double rz = dot(n, r, z);
    int it = 0;
    for (int k = 0; k < o->max_iter; k++) {
        if (o->rtol > 0 && sqrt(dot(n, r, r)) <= o->rtol * bnorm) break;
        if (rz == 0.0) break;
        orc_apply_op(cx, p, q);
        double pqk = dot(n, p, q);
        if (!(pqk > 0.0)) {
            status = ORC_ERR_BREAKDOWN;
            break;
        }
        if (hist) {
            memcpy(hist + (0L * (o->max_iter + 1) + k) * n, r, sizeof(double) * n);
            memcpy(hist + (1L * (o->max_iter + 1) + k) * n, z, sizeof(double) * n);
            memcpy(hist + (2L * (o->max_iter + 1) + k) * n, p, sizeof(double) * n);
            memcpy(hist + (3L * (o->max_iter + 1) + k) * n, q, sizeof(double) * n);
        }
        memcpy(newP + (long)k * n, p, sizeof(double) * n);
        memcpy(newQ + (long)k * n, q, sizeof(double) * n);
        newpq[k] = pqk;
        double alpha = rz / pqk;
        for (long i = 0; i < n; i++) {
            c[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        /* Residual replacement (not in the paper, which keeps the recurrence
         * residual of Algorithms 1-2 and warm-restarts from it in Algorithm 3):
         * after every N-th iteration the recurrence residual is replaced by the
         * true residual b - M c, from which z, the projection, (r, z) and beta
         * below follow; the stopping test and the next time step's warm
         * restart then see the true residual. */
        if (o->true_res_every > 0 && (k + 1) % o->true_res_every == 0) {
            orc_apply_op(cx, c, tmp);
            for (long i = 0; i < n; i++) r[i] = b[i] - tmp[i];
        }
        for (long i = 0; i < n; i++) z[i] = cx->invJ[i] * r[i];
        if (aug) {
            if (o->loop_mode == 0) {
                /* mu = (z, q_m)/(p_m, q_m): the printed denominator (p_m, p_m)
                 * is read as (p_m, q_m), the value that makes p_{k+1}
                 * M-conjugate to p_m. */
                const double *pm = P + (long)(kv - 1) * n, *qm = Q + (long)(kv - 1) * n;
                double mu = dot(n, z, qm) / pq[kv - 1];
                for (long i = 0; i < n; i++) z[i] -= mu * pm[i];
            } else {
                status = gram_coeffs(n, kv, P, Q, Q, z, tau);
                if (status) break;
                for (int j = 0; j < kv; j++)
                    for (long i = 0; i < n; i++) z[i] -= tau[j] * P[j * n + i];
            }
        }
        double rz_new = dot(n, r, z);
        double beta = rz_new / rz;
        for (long i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        rz = rz_new;
        it = k + 1;
    }
    if (hist && it <= o->max_iter) {
        memcpy(hist + (0L * (o->max_iter + 1) + it) * n, r, sizeof(double) * n);
        memcpy(hist + (1L * (o->max_iter + 1) + it) * n, z, sizeof(double) * n);
        memcpy(hist + (2L * (o->max_iter + 1) + it) * n, p, sizeof(double) * n);
    }
    /* Recycled basis for the next time step: the last min(it, kcap) directions. */
    if (status == ORC_OK && it > 0) {
        int keep = it < kcap ? it : kcap;
        for (int j = 0; j < keep; j++) {
            int src = it - keep + j;
            memcpy(P + (long)j * n, newP + (long)src * n, sizeof(double) * n);
            memcpy(Q + (long)j * n, newQ + (long)src * n, sizeof(double) * n);
            pq[j] = newpq[src];
        }
        *k_valid = keep;
    }
    memcpy(r_prev, r, sizeof(double) * n);
done:
    if (st) {
        st->iterations = it;
        st->bnorm = bnorm;
        st->rel_res = bnorm > 0 ? sqrt(dot(n, r, r)) / bnorm : 0.0;
        st->status = status;
    }
    free(b); free(r); free(z); free(p); free(q); free(tmp);
    free(newP); free(newQ); free(newpq);
    return status;
}

/* Dense assembly of M column by column (tiny grids only). */
void orc_dense_M(const orc_ctx *c, double *Mout)
{
    long n = c->n;
    double *e = calloc(n, sizeof(double)), *col = malloc(sizeof(double) * n);
    for (long j = 0; j < n; j++) {
        e[j] = 1.0;
        orc_apply_op(c, e, col);
        for (long i = 0; i < n; i++) Mout[i * n + j] = col[i];
        e[j] = 0.0;
    }
    free(e);
    free(col);
}
