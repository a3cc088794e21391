// fewha_conv3x3_fwd_tc: the learned warm start's 3x3 convolution on the
// 5th-generation tensor cores (tcgen05) of sm_103a, as an implicit GEMM with
// BF16 operands and FP32 accumulation in tensor memory (TMEM).  Not part of
// the paper's method (the network is a predictor of the warm start).
//
// One CTA computes two output rows y0, y0 + 1 (W <= 128 pixels) of one image
// for every output channel (two TMEM accumulators): D[x][co] = sum over taps (ky, kx) and input channels ci of
// in[ci][y+ky-1][x+kx-1] w[co][ci][ky][kx].
//   1. warp 0 allocates 64 TMEM columns (two 128 x N FP32 accumulators);
//   2. all threads stage the four input rows y0-1 .. y0+2 once in shared
//      memory as BF16, channel-minor: per (row, group of 8 channels) an array
//      of RP pixels of 16 bytes (8 channels), pixel q holding x = q - 1 (zero
//      for x outside the image and for padded channels), each 16-byte row
//      packed in registers and written with one store; and the weights as
//      per (tap, group of 8 input channels) the 8-row x 16-byte core matrices
//      of the output channels, read from w in its own (coalesced) order and
//      written value by value into a zeroed image;
//   3. one thread issues one tcgen05.mma (M = 128, N = Np, K = 16: two
//      channel groups) per output row, tap and channel-group pair: the A
//      operand of tap (ky, kx) for output row h is the staged row h + ky seen
//      from pixel kx on, a K-major matrix
//      without swizzle whose 8-pixel core matrices are 128 bytes apart
//      (stride-dimension offset) and whose channel groups are RP * 16 bytes
//      apart (leading-dimension offset), so no patch matrix is formed;
//      tcgen05.commit arrives on an mbarrier when they are done;
//   4. the CTA waits on the mbarrier (at most 0.5 s: on time-out it records
//      FEWHA_ERR_TIMEOUT, waits once more with the same limit, frees its TMEM
//      and returns); warps 4h..4h+3 read accumulator h, 32 lanes (pixels)
//      each, with tcgen05.ld, add the bias, apply ReLU and store; warp 0
//      frees the TMEM.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fewha.h"

namespace {

constexpr int kTcM = 128;       // output pixels per CTA (MMA M)
constexpr int kTcThreads = 256;
constexpr int kTcRows = 2;      // output rows per CTA (one accumulator of 32 TMEM columns each)
constexpr int kTcCols = 32 * kTcRows;  // TMEM columns allocated (a power of two >= 32)
constexpr unsigned long long kTcWaitNs = 500000000ull;  // a wait for the tensor cores gives up after 0.5 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (K-major, no swizzle): start address,
// leading-dimension byte offset (between core matrices adjacent along K),
// stride-dimension byte offset (between 8-row groups), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // version
    return d;                // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, BF16 A
// and B, both K-major, N = n, M = 128.
__device__ __forceinline__ uint32_t instr_desc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

constexpr int kRP = 136;  // staged pixels per (row, channel group): x = -1 .. 128 plus slack (multiple of 8)
// dynamic shared memory of the largest case (Cin 32, Cout 32): staged rows and weights
constexpr size_t kTcSmemCap = (size_t)(kTcRows + 2) * 4 * kRP * 16 + (size_t)9 * 4 * 4 * 128;

// 8 floats as 8 bfloat16 (round to nearest even) in one 16-byte word
__device__ __forceinline__ uint4 pack8(const float (&v)[8])
{
    uint4 u;
    __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]), p1 = __floats2bfloat162_rn(v[2], v[3]);
    __nv_bfloat162 p2 = __floats2bfloat162_rn(v[4], v[5]), p3 = __floats2bfloat162_rn(v[6], v[7]);
    u.x = *reinterpret_cast<unsigned int *>(&p0);
    u.y = *reinterpret_cast<unsigned int *>(&p1);
    u.z = *reinterpret_cast<unsigned int *>(&p2);
    u.w = *reinterpret_cast<unsigned int *>(&p3);
    return u;
}

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    const unsigned long long t0 = now_ns();
    for (unsigned it = 0;; it++) {
        if ((it & 63u) == 63u && now_ns() - t0 > kTcWaitNs) return false;
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

template <int NP>
__device__ __forceinline__ void tmem_load_row(uint32_t taddr, float (&v)[NP])
{
    uint32_t r[NP];
    if constexpr (NP == 16) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
              "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
              "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < NP; i++) v[i] = __uint_as_float(r[i]);
}

template <int NP>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_conv3x3_tc(const float *__restrict__ in, long in_bs, long in_cs, int Cin, const float *__restrict__ w,
                 const float *__restrict__ bias, float *__restrict__ out, long out_bs, long out_cs, int Cout, int H,
                 int W, int relu, int ncg, int *status)
{
    // ncg: groups of 8 input channels (even: Cin padded to a multiple of 16)
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int ty = (H + kTcRows - 1) / kTcRows;  // row tiles per image
    const int b = blockIdx.x / ty, y0 = (blockIdx.x - b * ty) * kTcRows;
    constexpr int SR = kTcRows + 2;                                // staged input rows y0-1 .. y0+kTcRows
    unsigned char *X = tc_smem;                                    // [SR][ncg][kRP] x 16 bytes
    unsigned char *Wt = tc_smem + (size_t)SR * ncg * kRP * 16;     // [9][ncg][NP / 8] core matrices of 128 bytes

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");

    // Every 16-byte row of a core matrix holds 8 consecutive input channels.
    // Weights, row (tap t, channel group g, output channel co): the image is
    // zeroed (padded channels stay 0), then w is read in its own order with
    // consecutive threads on consecutive floats (coalesced; the old per-row
    // gather touched a separate sector for every value) and each value is
    // written as bfloat16 to its place in the row.
    const int nb = NP >> 3;
    const int wvec = 9 * ncg * nb * 8;  // 16-byte words of the weight image
    for (int e = tid; e < wvec; e += kTcThreads) reinterpret_cast<uint4 *>(Wt)[e] = make_uint4(0u, 0u, 0u, 0u);
    // input: row (staged row r, channel group g, pixel q), q holding x = q - 1
    // and staged row r input row y0 + r - 1 (zero outside the image: the halo
    // pixels and rows beyond it); threads with consecutive pixels read
    // consecutive addresses of each channel, two rows of 8 channels at once
    const int nx = SR * ncg * kRP;
    for (int e0 = tid; e0 < nx; e0 += 2 * kTcThreads) {
        float v[2][8];
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int e = e0 + u * kTcThreads;
            const int r = e / (ncg * kRP), g = (e / kRP) % ncg, q = e % kRP;
            const int yy = y0 + r - 1, x = q - 1;
            const bool inside = e < nx && yy >= 0 && yy < H && x >= 0 && x < W;
            const float *px = in + (long)b * in_bs + (long)yy * W + x;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int ci = g * 8 + j;
                v[u][j] = (inside && ci < Cin) ? __ldg(px + (long)ci * in_cs) : 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int e = e0 + u * kTcThreads;
            if (e < nx) *reinterpret_cast<uint4 *>(X + (size_t)e * 16) = pack8(v[u]);
        }
    }
    __syncthreads();  // the weight image is zero
    {
        const int nw = Cout * Cin * 9;
        constexpr int UW = 8;  // loads in flight per thread
        for (int e0 = tid; e0 < nw; e0 += UW * kTcThreads) {
            float v[UW];
#pragma unroll
            for (int u = 0; u < UW; u++) {
                const int e = e0 + u * kTcThreads;
                v[u] = e < nw ? __ldg(w + e) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < UW; u++) {
                const int e = e0 + u * kTcThreads;
                if (e < nw) {
                    const int t = e % 9, cc = e / 9, ci = cc % Cin, co = cc / Cin;  // e = (co Cin + ci) 9 + t
                    unsigned char *row = Wt + (((t * ncg + (ci >> 3)) * nb + (co >> 3)) * 128 + (co & 7) * 16);
                    reinterpret_cast<__nv_bfloat16 *>(row)[ci & 7] = __float2bfloat16_rn(v[u]);
                }
            }
        }
    }
    // the operands become visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = tmem_base;

    if (tid == 0) {
        const uint32_t x0 = smem_u32(X), w0 = smem_u32(Wt), idesc = instr_desc(NP);
        for (int h = 0; h < kTcRows; h++) {  // output row y0 + h into TMEM columns 32 h ..
            int acc = 0;
            for (int t = 0; t < 9; t++) {
                const int ky = t / 3, kx = t - ky * 3;
                for (int j = 0; j < ncg; j += 2) {
                    // A: staged row h + ky, channel groups j, j+1, pixels kx .. kx + 127
                    const uint64_t ad =
                        smem_desc(x0 + (uint32_t)((((h + ky) * ncg + j) * kRP + kx) * 16), kRP * 16u, 128u);
                    // B: tap t, channel groups j, j+1, all output channels
                    const uint64_t bd =
                        smem_desc(w0 + (uint32_t)((t * ncg + j) * (NP >> 3) * 128), (NP >> 3) * 128u, 128u);
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(taddr + 32u * h),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                    acc = 1;
                }
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&mbar))
                     : "memory");
    }
    __shared__ int ok_all;
    if (tid == 0) ok_all = 1;
    __syncthreads();
    bool ok = mbar_wait(smem_u32(&mbar), 0);
    if (!ok) ok_all = 0;
    __syncthreads();
    if (!ok_all) {
        // the MMAs did not complete in time: record it, give them one more
        // bounded wait, then free the TMEM and return
        if (tid == 0 && status) atomicCAS(status, 0, FEWHA_ERR_TIMEOUT);
        mbar_wait(smem_u32(&mbar), 0);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTcCols)
                         : "memory");
        return;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp < 4 * kTcRows) {
        // warps 4h .. 4h+3: accumulator h (output row y0 + h); its row m =
        // 32 (warp % 4) + lane (pixel x = m) lives in TMEM lane m
        const int h = warp >> 2, y = y0 + h;
        float v[NP];
        tmem_load_row<NP>(taddr + 32u * h + ((uint32_t)((warp & 3) * 32) << 16), v);
        const int x = (warp & 3) * 32 + (tid & 31);
        if (x < W && y < H) {
#pragma unroll
            for (int co = 0; co < NP; co++) {
                if (co < Cout) {
                    float r = v[co] + (bias ? bias[co] : 0.f);
                    if (relu) r = r > 0.f ? r : 0.f;
                    out[(long)b * out_bs + (long)co * out_cs + (long)y * W + x] = r;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTcCols) : "memory");
}

}  // namespace

extern "C" int fewha_conv3x3_fwd_tc(const float *in, long in_bs, long in_cs, int Cin, const float *w,
                                    const float *bias, float *out, long out_bs, long out_cs, int Cout, int B, int H,
                                    int W, int relu, int *status_dev, cudaStream_t s)
{
    if (!in || !w || !out || Cin < 1 || Cin > 32 || Cout < 1 || Cout > 32 || B < 1 || H < 1 || W < 1 || W > kTcM)
        return FEWHA_ERR_ARG;
    const long nrt = (H + kTcRows - 1) / kTcRows;  // row tiles per image
    if ((long)B * nrt > 0x7FFFFFFFL) return FEWHA_ERR_ARG;
    const int ncg = (Cin + 15) / 16 * 2;  // groups of 8 input channels, an even number
    const int np = Cout <= 16 ? 16 : 32;
    // staged rows and weights; the MMAs read only inside them (the last A
    // view ends at pixel 2 + 127 < kRP of row 2)
    const size_t smem = (size_t)(kTcRows + 2) * ncg * kRP * 16 + (size_t)9 * ncg * (np / 8) * 128;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FEWHA_ERR_CUDA;
    // the shared-memory attribute is raised once per device and variant (a
    // host call per launch would leave the GPU idle between short launches)
    auto launch = [&](auto kern, size_t *done) {
        cudaError_t e = cudaSuccess;
        if (done[dev] < smem) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemCap);
            if (e == cudaSuccess) done[dev] = kTcSmemCap;
        }
        if (e == cudaSuccess)
            kern<<<(unsigned)(B * nrt), kTcThreads, smem, s>>>(in, in_bs, in_cs, Cin, w, bias, out, out_bs, out_cs, Cout,
                                                            H, W, relu, ncg, status_dev);
        return e;
    };
    static size_t set16[64], set32[64];
    cudaError_t e;
    if (np == 16)
        e = launch(k_conv3x3_tc<16>, set16);
    else
        e = launch(k_conv3x3_tc<32>, set32);
    if (e != cudaSuccess) return FEWHA_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? FEWHA_OK : FEWHA_ERR_CUDA;
}
