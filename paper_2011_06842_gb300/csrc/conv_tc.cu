// fewha_conv3x3_fwd_tc: the learned warm start's 3x3 convolution on the
// 5th-generation tensor cores (tcgen05) of sm_103a, as an implicit GEMM
//     out[p][co] = sum_k A[p][k] B[co][k],   k = ci * 9 + tap,
// A the image patches (im2col) of 128 output pixels, B the weights, with
// BF16 operands and FP32 accumulation in tensor memory (TMEM).  Not part of
// the paper's method (the network is a predictor of the warm start).
//
// One CTA computes 128 consecutive output pixels of one image for every
// output channel:
//   1. warp 0 allocates 32 TMEM columns (the 128 x N FP32 accumulator);
//   2. all threads write A (128 x Kp) and B (Np x Kp) into shared memory as
//      BF16 in the canonical K-major layout without swizzle: 8-row x 16-byte
//      core matrices, the core matrices of one 8-row group adjacent along K
//      (128 bytes apart, the descriptor's leading-dimension offset), the
//      8-row groups Kp / 8 * 128 bytes apart (its stride-dimension offset);
//   3. one thread issues Kp / 16 tcgen05.mma (M = 128, N = Np, K = 16 each)
//      and tcgen05.commit arrives on an mbarrier when they are done;
//   4. the CTA waits on the mbarrier (at most 0.5 s: on time-out it records
//      FEWHA_ERR_TIMEOUT, waits once more with the same limit, frees its TMEM
//      and returns); warps 0-3 read their 32 accumulator lanes each with
//      tcgen05.ld, add the bias, apply ReLU and store; warp 0 frees the TMEM.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fewha.h"

namespace {

constexpr int kTcM = 128;       // output pixels per CTA (MMA M)
constexpr int kTcThreads = 256;
constexpr int kTcCols = 32;     // TMEM columns allocated (>= Np, a power of two >= 32)
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

// Byte offset of element (row, k) in the canonical layout of a rows x kp tile.
__device__ __forceinline__ int tile_off(int row, int k, int kp)
{
    return (row >> 3) * (kp >> 3) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
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
                 int W, int relu, int kp, int *status)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const long hw = (long)H * W;
    const int tiles = (int)((hw + kTcM - 1) / kTcM);
    const int b = blockIdx.x / tiles;
    const long p0 = (long)(blockIdx.x - b * tiles) * kTcM;
    unsigned char *A = tc_smem;                       // kTcM x kp BF16
    unsigned char *Bm = tc_smem + (size_t)kTcM * kp * 2;  // NP x kp BF16

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");

    // B: weights w[co][ci][tap] at k = ci * 9 + tap, zero-padded to NP x kp
    const int K = Cin * 9;
    for (int e = tid; e < NP * kp; e += kTcThreads) {
        const int n = e / kp, k = e - n * kp;
        const float v = (n < Cout && k < K) ? w[(long)n * K + k] : 0.f;
        *reinterpret_cast<__nv_bfloat16 *>(Bm + tile_off(n, k, kp)) = __float2bfloat16_rn(v);
    }
    // A: patches; consecutive threads take consecutive pixels of one (ci, tap)
    for (int e = tid; e < kTcM * kp; e += kTcThreads) {
        const int k = e / kTcM, m = e - k * kTcM;
        const long p = p0 + m;
        float v = 0.f;
        if (k < K && p < hw) {
            const int ci = k / 9, tap = k - ci * 9;
            const int y = (int)(p / W) + tap / 3 - 1, x = (int)(p % W) + tap % 3 - 1;
            if (y >= 0 && y < H && x >= 0 && x < W) v = in[(long)b * in_bs + (long)ci * in_cs + (long)y * W + x];
        }
        *reinterpret_cast<__nv_bfloat16 *>(A + tile_off(m, k, kp)) = __float2bfloat16_rn(v);
    }
    // the tiles become visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = tmem_base;

    if (tid == 0) {
        const uint32_t a0 = smem_u32(A), b0 = smem_u32(Bm), sbo = (uint32_t)(kp >> 3) * 128u;
        const uint32_t idesc = instr_desc(NP);
        for (int ks = 0; ks < kp / 16; ks++) {
            const uint64_t ad = smem_desc(a0 + (uint32_t)ks * 256u, 128u, sbo);
            const uint64_t bd = smem_desc(b0 + (uint32_t)ks * 256u, 128u, sbo);
            const uint32_t acc = ks > 0 ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(taddr),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
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
    if (warp < 4) {
        // accumulator row m = 32 warp + lane lives in TMEM lane m
        float v[NP];
        tmem_load_row<NP>(taddr + ((uint32_t)(warp * 32) << 16), v);
        const long p = p0 + warp * 32 + (tid & 31);
        if (p < hw) {
#pragma unroll
            for (int co = 0; co < NP; co++) {
                if (co < Cout) {
                    float r = v[co] + (bias ? bias[co] : 0.f);
                    if (relu) r = r > 0.f ? r : 0.f;
                    out[(long)b * out_bs + (long)co * out_cs + p] = r;
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
    if (!in || !w || !out || Cin < 1 || Cin > 32 || Cout < 1 || Cout > 32 || B < 1 || H < 1 || W < 1)
        return FEWHA_ERR_ARG;
    const int kp = (Cin * 9 + 15) / 16 * 16;
    const long tiles = ((long)H * W + kTcM - 1) / kTcM;
    if (tiles * B > 0x7FFFFFFFL) return FEWHA_ERR_ARG;
    const size_t smem = (size_t)kTcM * kp * 2 + (size_t)(Cout <= 16 ? 16 : 32) * kp * 2;
    cudaError_t e;
    if (Cout <= 16) {
        e = cudaFuncSetAttribute(k_conv3x3_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            k_conv3x3_tc<16><<<(unsigned)(tiles * B), kTcThreads, smem, s>>>(in, in_bs, in_cs, Cin, w, bias, out,
                                                                            out_bs, out_cs, Cout, H, W, relu, kp,
                                                                            status_dev);
    } else {
        e = cudaFuncSetAttribute(k_conv3x3_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            k_conv3x3_tc<32><<<(unsigned)(tiles * B), kTcThreads, smem, s>>>(in, in_bs, in_cs, Cin, w, bias, out,
                                                                            out_bs, out_cs, Cout, H, W, relu, kp,
                                                                            status_dev);
    }
    if (e != cudaSuccess) return FEWHA_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? FEWHA_OK : FEWHA_ERR_CUDA;
}
