// Kernels of the learned warm start: a small convolutional network over the
// previous frames' layer coefficients (3x3 convolutions, zero padding, ReLU),
// its backward pass, the MSE loss and the Adam update.  FP32, NCHW tensors
// with an explicit batch stride (the layers of one size are a batch).
// Not part of the paper's method: a predictor of the next time step's warm
// start and deflation directions; PCG stays the solver.
#include <cuda_runtime.h>

#include "../../include/fewha.h"

namespace {

constexpr int TX = 16;    // output tile width
constexpr int TY = 32;    // output tile height (two rows per thread)
constexpr int CO_T = 8;   // output channels per block
constexpr int CI_T = 8;   // input channels staged per step
constexpr int NT = TX * TY / 2;

// out[b][co][y][x] = act(bias[co] + sum_ci sum_{ky,kx} w[co][ci][ky][kx] in[b][ci][y+ky-1][x+kx-1])
// (zero outside the image).  Tensors are addressed as base + b*bs + c*cs + y*W + x.
// For the data gradient the weights are read transposed and flipped
// (wt_mode = 1: w[ci][co][2-ky][2-kx] of a Cin x Cout tensor).  Each thread
// computes two vertically adjacent pixels for CO_T channels; the weights of
// one (input channel, tap) are staged as CO_T consecutive floats so that a
// thread reads them with two 16-byte shared loads.
__global__ void __launch_bounds__(NT) k_conv3x3(const float *__restrict__ in, long in_bs, long in_cs, int Cin,
                                                const float *__restrict__ w, const float *__restrict__ bias,
                                                float *__restrict__ out, long out_bs, long out_cs, int Cout, int H,
                                                int W, int relu, int wt_mode)
{
    __shared__ float tile[CI_T][TY + 2][TX + 2];
    __shared__ __align__(16) float wsh[CI_T][9][CO_T];
    const int tx = threadIdx.x % TX, ty2 = (threadIdx.x / TX) * 2;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int nco = (Cout + CO_T - 1) / CO_T;
    const int b = blockIdx.z / nco, co0 = (blockIdx.z % nco) * CO_T;
    const float *inb = in + (long)b * in_bs;
    float acc0[CO_T], acc1[CO_T];
#pragma unroll
    for (int j = 0; j < CO_T; j++) acc0[j] = acc1[j] = (bias && co0 + j < Cout) ? bias[co0 + j] : 0.f;
    for (int ci0 = 0; ci0 < Cin; ci0 += CI_T) {
        for (int e = threadIdx.x; e < CI_T * (TY + 2) * (TX + 2); e += NT) {
            const int c = e / ((TY + 2) * (TX + 2)), r = (e / (TX + 2)) % (TY + 2), q = e % (TX + 2);
            const int y = y0 + r - 1, x = x0 + q - 1;
            float v = 0.f;
            if (ci0 + c < Cin && y >= 0 && y < H && x >= 0 && x < W) v = inb[(long)(ci0 + c) * in_cs + (long)y * W + x];
            tile[c][r][q] = v;
        }
        for (int e = threadIdx.x; e < CO_T * CI_T * 9; e += NT) {
            const int c = e / (9 * CO_T), k = (e / CO_T) % 9, j = e % CO_T;
            const int co = co0 + j, ci = ci0 + c;
            float v = 0.f;
            if (co < Cout && ci < Cin)
                v = wt_mode ? w[((long)ci * Cout + co) * 9 + (8 - k)] : w[((long)co * Cin + ci) * 9 + k];
            wsh[c][k][j] = v;
        }
        __syncthreads();
#pragma unroll 2
        for (int c = 0; c < CI_T; c++) {
            float v[4][3];
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int q = 0; q < 3; q++) v[r][q] = tile[c][ty2 + r][tx + q];
#pragma unroll
            for (int k = 0; k < 9; k++) {
                const float4 wa = *reinterpret_cast<const float4 *>(&wsh[c][k][0]);
                const float4 wb = *reinterpret_cast<const float4 *>(&wsh[c][k][4]);
                const float wk[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
                const float a = v[k / 3][k % 3], d = v[k / 3 + 1][k % 3];
#pragma unroll
                for (int j = 0; j < CO_T; j++) {
                    acc0[j] += wk[j] * a;
                    acc1[j] += wk[j] * d;
                }
            }
        }
        __syncthreads();
    }
    const int x = x0 + tx;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int y = y0 + ty2 + h;
        if (x < W && y < H)
#pragma unroll
            for (int j = 0; j < CO_T; j++)
                if (co0 + j < Cout) {
                    float v = h ? acc1[j] : acc0[j];
                    if (relu) v = v > 0.f ? v : 0.f;
                    out[(long)b * out_bs + (long)(co0 + j) * out_cs + (long)y * W + x] = v;
                }
    }
}

// Partial weight/bias gradients of one (batch, spatial tile): thread t owns
// weight entries t, t + 256, ... of the Cout x Cin x 9 tensor.
constexpr int TS = 16;  // spatial tile of the weight gradient

__global__ void __launch_bounds__(TS *TS) k_conv3x3_wgrad_partial(const float *__restrict__ in, long in_bs, long in_cs,
                                                                 int Cin, const float *__restrict__ gout, long gout_bs,
                                                                 long gout_cs, int Cout, int H, int W,
                                                                 float *__restrict__ part)
{
    extern __shared__ float sm[];
    float *tin = sm;                                // [Cin][TS+2][TS+2]
    float *tg = sm + Cin * (TS + 2) * (TS + 2);     // [Cout][TS][TS]
    const int tiles_x = (W + TS - 1) / TS, tiles_y = (H + TS - 1) / TS;
    const int tile = blockIdx.x % (tiles_x * tiles_y), b = blockIdx.x / (tiles_x * tiles_y);
    const int x0 = (tile % tiles_x) * TS, y0 = (tile / tiles_x) * TS;
    for (int e = threadIdx.x; e < Cin * (TS + 2) * (TS + 2); e += blockDim.x) {
        const int c = e / ((TS + 2) * (TS + 2)), r = (e / (TS + 2)) % (TS + 2), q = e % (TS + 2);
        const int y = y0 + r - 1, x = x0 + q - 1;
        tin[e] = (y >= 0 && y < H && x >= 0 && x < W) ? in[(long)b * in_bs + (long)c * in_cs + (long)y * W + x] : 0.f;
    }
    for (int e = threadIdx.x; e < Cout * TS * TS; e += blockDim.x) {
        const int c = e / (TS * TS), r = (e / TS) % TS, q = e % TS;
        const int y = y0 + r, x = x0 + q;
        tg[e] = (y < H && x < W) ? gout[(long)b * gout_bs + (long)c * gout_cs + (long)y * W + x] : 0.f;
    }
    __syncthreads();
    const int nw = Cout * Cin * 9;
    float *dst = part + (long)blockIdx.x * (nw + Cout);
    for (int e = threadIdx.x; e < nw; e += blockDim.x) {
        const int co = e / (Cin * 9), ci = (e / 9) % Cin, k = e % 9, ky = k / 3, kx = k % 3;
        const float *g = tg + co * TS * TS;
        const float *t = tin + ci * (TS + 2) * (TS + 2) + ky * (TS + 2) + kx;
        float a = 0.f;
        for (int r = 0; r < TS; r++)
#pragma unroll 4
            for (int q = 0; q < TS; q++) a += g[r * TS + q] * t[r * (TS + 2) + q];
        dst[e] = a;
    }
    for (int co = threadIdx.x; co < Cout; co += blockDim.x) {
        float a = 0.f;
        for (int e = 0; e < TS * TS; e++) a += tg[co * TS * TS + e];
        dst[nw + co] = a;
    }
}

// Sum of the per-tile partials in tile order (deterministic); accumulate
// adds to the gradients already stored.
__global__ void k_reduce_partials(const float *__restrict__ part, int nparts, int len, float *__restrict__ gw,
                                  float *__restrict__ gb, int nw, int accumulate)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int p = 0; p < nparts; p++) a += part[(long)p * len + e];
        float *dst = e < nw ? gw + e : gb + (e - nw);
        *dst = accumulate ? *dst + (float)a : (float)a;
    }
}

__global__ void k_relu_bwd(const float *__restrict__ act, float *__restrict__ g, long n)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        if (!(act[i] > 0.f)) g[i] = 0.f;
}

// grad = 2 (pred - target) / n; per-block partial sums of (pred - target)^2.
__global__ void k_mse(const float *__restrict__ pred, const float *__restrict__ target, float *__restrict__ grad,
                      long n, float inv_n, double *__restrict__ loss_part)
{
    __shared__ double sh[256];
    double a = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float d = pred[i] - target[i];
        grad[i] = 2.f * d * inv_n;
        a += (double)d * d;
    }
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = sh[0];
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       long n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// y = x * sqrt(s) (mode 0), x / sqrt(s) (mode 1), y += x / sqrt(s) (mode 2)
__global__ void k_scale(const float *__restrict__ x, const float *__restrict__ sc, float *__restrict__ y, long n,
                        int mode)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float r = sqrtf(sc[i]);
        if (mode == 0)
            y[i] = x[i] * r;
        else if (mode == 1)
            y[i] = x[i] / r;
        else
            y[i] += x[i] / r;
    }
}

// Training targets of the network (channel stride n): t0 = (c_next - c_cur) * sqrt(s);
// t_k = t0 where group[i] == k, else 0 (k = 1..4, the wavelet scale groups).
__global__ void k_targets(const float *__restrict__ c_next, const float *__restrict__ c_cur,
                          const float *__restrict__ sc, const signed char *__restrict__ group, float *__restrict__ t,
                          long n)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float d = (c_next[i] - c_cur[i]) * sqrtf(sc[i]);
        const int g = group[i];
        t[i] = d;
#pragma unroll
        for (int k = 1; k <= 4; k++) t[k * n + i] = (g == k) ? d : 0.f;
    }
}

// --- deflated warm start: Galerkin correction over predicted directions ----
constexpr int kMaxDir = FEWHA_MAX_DEFLATE;
constexpr int kChunks = 32;

// r0 = (b - b_prev) + r_prev (the warm restart of Algorithm 3)
__global__ void k_warm_residual(const float *__restrict__ b, const float *__restrict__ b_prev,
                                const float *__restrict__ r_prev, float *__restrict__ r0, long n)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        r0[i] = (b[i] - b_prev[i]) + r_prev[i];
}

struct DotPairs {
    const float *x[64], *y[64];
};

// part[p * kChunks + chunk] = partial (x_p, y_p) over one chunk (FP32 per
// thread, FP64 across the block; fixed order, deterministic).
__global__ void __launch_bounds__(256) k_dots(const __grid_constant__ DotPairs P, long n, double *__restrict__ part)
{
    __shared__ double sh[8];
    const int p = blockIdx.x, chunk = blockIdx.y;
    const long per = (n + kChunks - 1) / kChunks, lo = chunk * per, hi = min(n, lo + per);
    const float *x = P.x[p], *y = P.y[p];
    float a = 0.f;
    for (long i = lo + threadIdx.x; i < hi; i += blockDim.x) a += x[i] * y[i];
    double d = a;
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
        part[p * kChunks + chunk] = t;
    }
}

// One thread: G = sym(D^T Q), g = D^T r0, Cholesky of G with directions whose
// pivot falls below 1e-10 of their diagonal dropped, w = G^{-1} g;
// ||r0 - Q w||^2 = (r0,r0) - 2 w.(Q^T r0) + w^T (Q^T Q) w.  The correction is
// taken when that is below (r0, r0).
// info: [0] taken, [1] ||r0 - Q w||, [2] ||r0||, [3] kept directions, [4..4+nd) w
__global__ void k_deflate_solve(const double *__restrict__ part, int nd, double *__restrict__ info,
                                float *__restrict__ wf)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    auto sum = [&](int p) {
        double t = 0.0;
        for (int c = 0; c < kChunks; c++) t += part[p * kChunks + c];
        return t;
    };
    // pair order: (d_i, r0) i; (d_i, q_j) i,j; (q_i, r0) i; (q_i, q_j) i,j; (r0, r0)
    double G[kMaxDir][kMaxDir], QQ[kMaxDir][kMaxDir], g[kMaxDir], qr[kMaxDir], L[kMaxDir][kMaxDir], w[kMaxDir];
    int keep[kMaxDir];
    int p = 0;
    for (int i = 0; i < nd; i++) g[i] = sum(p++);
    for (int i = 0; i < nd; i++)
        for (int j = 0; j < nd; j++) G[i][j] = sum(p++);
    for (int i = 0; i < nd; i++) qr[i] = sum(p++);
    for (int i = 0; i < nd; i++)
        for (int j = 0; j < nd; j++) QQ[i][j] = sum(p++);
    const double rr = sum(p++);
    int kept = 0;
    for (int j = 0; j < nd; j++) {
        keep[j] = 0;
        double d = 0.5 * (G[j][j] + G[j][j]);
        const double dj = d;
        for (int k = 0; k < j; k++)
            if (keep[k]) d -= L[j][k] * L[j][k];
        if (!(dj > 0.0) || !(d > 1e-10 * dj)) {
            for (int k = 0; k <= j; k++) L[j][k] = 0.0;
            continue;
        }
        keep[j] = 1;
        kept++;
        L[j][j] = sqrt(d);
        for (int i = j + 1; i < nd; i++) {
            double v = 0.5 * (G[i][j] + G[j][i]);
            for (int k = 0; k < j; k++)
                if (keep[k]) v -= L[i][k] * L[j][k];
            L[i][j] = v / L[j][j];
        }
    }
    double y[kMaxDir];
    for (int i = 0; i < nd; i++) {
        y[i] = 0.0;
        if (!keep[i]) continue;
        double v = g[i];
        for (int k = 0; k < i; k++)
            if (keep[k]) v -= L[i][k] * y[k];
        y[i] = v / L[i][i];
    }
    for (int i = nd - 1; i >= 0; i--) {
        w[i] = 0.0;
        if (!keep[i]) continue;
        double v = y[i];
        for (int k = i + 1; k < nd; k++)
            if (keep[k]) v -= L[k][i] * w[k];
        w[i] = v / L[i][i];
    }
    double rr1 = rr;
    for (int i = 0; i < nd; i++) {
        rr1 -= 2.0 * w[i] * qr[i];
        for (int j = 0; j < nd; j++) rr1 += w[i] * QQ[i][j] * w[j];
    }
    bool ok = kept > 0 && rr1 < rr && rr1 == rr1;
    for (int i = 0; i < nd; i++) ok = ok && (w[i] == w[i]);
    info[0] = ok ? 1.0 : 0.0;
    info[1] = sqrt(fmax(rr1, 0.0));
    info[2] = sqrt(rr);
    info[3] = kept;
    for (int i = 0; i < nd; i++) {
        info[4 + i] = w[i];
        wf[i] = (float)w[i];
    }
}

// If taken: c += D w, r_prev <- r0 - Q w, b_prev <- b.
__global__ void k_deflate_update(const double *__restrict__ info, const float *__restrict__ wf, int nd,
                                 const float *__restrict__ D, long ldd, const float *__restrict__ Q, long ldq,
                                 const float *__restrict__ b, const float *__restrict__ r0, float *__restrict__ c,
                                 float *__restrict__ b_prev, float *__restrict__ r_prev, long n)
{
    // not taken: the plain warm restart r0 is folded into the state
    const bool taken = info[0] != 0.0;
    if (!taken) {
        for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
            r_prev[i] = r0[i];
            b_prev[i] = b[i];
        }
        return;
    }
    float w[kMaxDir];
#pragma unroll
    for (int j = 0; j < kMaxDir; j++) w[j] = j < nd ? wf[j] : 0.f;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        float cv = c[i], rv = r0[i];
        for (int j = 0; j < nd; j++) {
            cv += w[j] * D[j * ldd + i];
            rv -= w[j] * Q[j * ldq + i];
        }
        c[i] = cv;
        r_prev[i] = rv;
        b_prev[i] = b[i];
    }
}

int ck() { return cudaGetLastError() == cudaSuccess ? FEWHA_OK : FEWHA_ERR_CUDA; }

}  // namespace

extern "C" {

int fewha_conv3x3_fwd(const float *in, long in_bs, long in_cs, int Cin, const float *w, const float *bias,
                      float *out, long out_bs, long out_cs, int Cout, int B, int H, int W, int relu, cudaStream_t s)
{
    if (!in || !w || !out || Cin < 1 || Cout < 1 || B < 1 || H < 1 || W < 1) return FEWHA_ERR_ARG;
    dim3 grid((W + TX - 1) / TX, (H + TY - 1) / TY, B * ((Cout + CO_T - 1) / CO_T));
    if (grid.z > 65535) return FEWHA_ERR_ARG;
    k_conv3x3<<<grid, NT, 0, s>>>(in, in_bs, in_cs, Cin, w, bias, out, out_bs, out_cs, Cout, H, W, relu, 0);
    return ck();
}

int fewha_conv3x3_bwd_data(const float *gout, long gout_bs, long gout_cs, int Cout, const float *w, float *gin,
                           long gin_bs, long gin_cs, int Cin, int B, int H, int W, cudaStream_t s)
{
    if (!gout || !w || !gin || Cin < 1 || Cout < 1 || B < 1 || H < 1 || W < 1) return FEWHA_ERR_ARG;
    dim3 grid((W + TX - 1) / TX, (H + TY - 1) / TY, B * ((Cin + CO_T - 1) / CO_T));
    if (grid.z > 65535) return FEWHA_ERR_ARG;
    k_conv3x3<<<grid, NT, 0, s>>>(gout, gout_bs, gout_cs, Cout, w, nullptr, gin, gin_bs, gin_cs, Cin, H, W, 0, 1);
    return ck();
}

long fewha_conv3x3_wgrad_workspace(int Cin, int Cout, int B, int H, int W)
{
    if (Cin < 1 || Cout < 1 || B < 1 || H < 1 || W < 1) return 0;
    const long tiles = (long)((W + TS - 1) / TS) * ((H + TS - 1) / TS) * B;
    return tiles * ((long)Cout * Cin * 9 + Cout);
}

int fewha_conv3x3_bwd_weight(const float *in, long in_bs, long in_cs, int Cin, const float *gout, long gout_bs,
                             long gout_cs, int Cout, int B, int H, int W, float *gw, float *gb, int accumulate,
                             float *workspace, cudaStream_t s)
{
    if (!in || !gout || !gw || !gb || !workspace || Cin < 1 || Cout < 1 || B < 1 || H < 1 || W < 1)
        return FEWHA_ERR_ARG;
    const long tiles = (long)((W + TS - 1) / TS) * ((H + TS - 1) / TS) * B;
    const size_t smem = ((size_t)Cin * (TS + 2) * (TS + 2) + (size_t)Cout * TS * TS) * sizeof(float);
    if (smem > 200 * 1024 || tiles > 0x7fffffffL) return FEWHA_ERR_ARG;
    if (cudaFuncSetAttribute(k_conv3x3_wgrad_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return FEWHA_ERR_CUDA;
    k_conv3x3_wgrad_partial<<<(unsigned)tiles, TS * TS, smem, s>>>(in, in_bs, in_cs, Cin, gout, gout_bs, gout_cs,
                                                                   Cout, H, W, workspace);
    const int len = Cout * Cin * 9 + Cout;
    k_reduce_partials<<<(len + 255) / 256, 256, 0, s>>>(workspace, (int)tiles, len, gw, gb, Cout * Cin * 9,
                                                         accumulate);
    return ck();
}

int fewha_relu_bwd(const float *act, float *g, long n, cudaStream_t s)
{
    if (!act || !g || n < 0) return FEWHA_ERR_ARG;
    k_relu_bwd<<<512, 256, 0, s>>>(act, g, n);
    return ck();
}

int fewha_mse_grad(const float *pred, const float *target, float *grad, long n, double *loss_part512, cudaStream_t s)
{
    if (!pred || !target || !grad || !loss_part512 || n < 1) return FEWHA_ERR_ARG;
    k_mse<<<512, 256, 0, s>>>(pred, target, grad, n, 1.f / (float)n, loss_part512);
    return ck();
}

int fewha_adam_step(float *param, const float *grad, float *m, float *v, long n, float lr, float beta1, float beta2,
                    float eps, int step, cudaStream_t s)
{
    if (!param || !grad || !m || !v || n < 1 || step < 1) return FEWHA_ERR_ARG;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    k_adam<<<512, 256, 0, s>>>(param, grad, m, v, n, lr, beta1, beta2, eps, c1, c2);
    return ck();
}

int fewha_scale(const float *x, const float *s_, float *y, long n, int mode, cudaStream_t s)
{
    if (!x || !s_ || !y || n < 1 || mode < 0 || mode > 2) return FEWHA_ERR_ARG;
    k_scale<<<512, 256, 0, s>>>(x, s_, y, n, mode);
    return ck();
}

int fewha_learned_targets(const float *c_next, const float *c_cur, const float *scale, const signed char *group,
                          float *targets5, long n, cudaStream_t s)
{
    if (!c_next || !c_cur || !scale || !group || !targets5 || n < 1) return FEWHA_ERR_ARG;
    k_targets<<<512, 256, 0, s>>>(c_next, c_cur, scale, group, targets5, n);
    return ck();
}

int fewha_deflate_warm_start(const float *b, const float *D, long ldd, const float *Q, long ldq, int nd, float *c,
                             float *b_prev, float *r_prev, long n, float *r0_work, double *work, double *info,
                             cudaStream_t s)
{
    if (!b || !D || !Q || !c || !b_prev || !r_prev || !r0_work || !work || !info || n < 1 || nd < 1 ||
        nd > kMaxDir || ldd < n || ldq < n)
        return FEWHA_ERR_ARG;
    static_assert(2 * kMaxDir + kMaxDir * kMaxDir <= 64 && kMaxDir * kMaxDir + 1 <= 64, "dot pairs per launch");
    static_assert((2 * kMaxDir + 2 * kMaxDir * kMaxDir + 1) * kChunks <= FEWHA_DEFLATE_WORK_DOUBLES, "work");
    static_assert(4 + kMaxDir + (kMaxDir + 1) / 2 <= FEWHA_DEFLATE_INFO_DOUBLES, "info");
    k_warm_residual<<<512, 256, 0, s>>>(b, b_prev, r_prev, r0_work, n);
    DotPairs P;
    int p = 0;
    for (int i = 0; i < nd; i++) P.x[p] = D + i * ldd, P.y[p++] = r0_work;
    for (int i = 0; i < nd; i++)
        for (int j = 0; j < nd; j++) P.x[p] = D + i * ldd, P.y[p++] = Q + j * ldq;
    for (int i = 0; i < nd; i++) P.x[p] = Q + i * ldq, P.y[p++] = r0_work;
    // (q_i, q_j) and (r0, r0) go in a second launch (at most 64 pairs each)
    DotPairs P2;
    int p2 = 0;
    for (int i = 0; i < nd; i++)
        for (int j = 0; j < nd; j++) P2.x[p2] = Q + i * ldq, P2.y[p2++] = Q + j * ldq;
    P2.x[p2] = r0_work, P2.y[p2++] = r0_work;
    k_dots<<<dim3(p, kChunks), 256, 0, s>>>(P, n, work);
    k_dots<<<dim3(p2, kChunks), 256, 0, s>>>(P2, n, work + (long)p * kChunks);
    float *wf = reinterpret_cast<float *>(info + 4 + kMaxDir);
    k_deflate_solve<<<1, 32, 0, s>>>(work, nd, info, wf);
    k_deflate_update<<<512, 256, 0, s>>>(info, wf, nd, D, ldd, Q, ldq, b, r0_work, c, b_prev, r_prev, n);
    return ck();
}

}  // extern "C"
