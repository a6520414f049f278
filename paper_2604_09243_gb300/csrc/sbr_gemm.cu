// sbr_gemm.cu -- BF16 tensor-core GEMM on the 5th-generation tensor cores
// (tcgen05) for the learned surrogate: C = A B^T with A [M x K] and B [N x K]
// both K-contiguous BF16, FP32 accumulation in tensor memory (TMEM).
//
// One CTA of 128 threads computes a 128 x BN tile (BN = 128, or 64 when the
// 128-wide grid would leave SMs idle):
//   - warp 0 (one lane) streams 128 x 64 tiles of A and BN x 64 tiles of B
//     into shared memory with TMA (cp.async.bulk.tensor, 128-byte swizzle)
//     through a 3-stage ring of mbarriers, refilling a stage once the MMAs
//     that read it have completed;
//   - warp 1 (one lane) issues tcgen05.mma (M = 128, N = BN, K = 16 per
//     instruction, 4 per stage) as soon as a stage lands and commits each
//     stage back to the producer, so MMA issue never waits for a refill;
//   - after the last K step all four warps read the accumulator out of TMEM
//     with tcgen05.ld (warp w owns rows 32w .. 32w + 31), apply the fused
//     epilogue (bias, GELU, GELU derivative) into the now idle pipeline
//     buffers, and write the tile out row by row with coalesced 16-byte stores
//     (the pre-activation read of the GELU-derivative epilogue is staged the
//     same way).
// Every wait is bounded: on a timeout the CTA records an error flag, skips the
// remaining work, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>

#include "sbr_internal.h"

namespace sbr {

namespace {

constexpr int kBM = 128, kBK = 64, kStages = 3;  // 3 stages keep a CTA at ~103 KB: two per SM
constexpr int kTileA = kBM * kBK * 2;  // bytes
constexpr unsigned kSpin = 1u << 24;  // try_wait rounds before a wait gives up
template <int BN>
struct Cfg {
    static constexpr int kTileB = BN * kBK * 2;
    static constexpr int kStageBytes = kTileA + kTileB;
    static constexpr int kPipe = kStages * kStageBytes;
    // epilogue staging (reuses the pipeline buffers): FP32 [128][BN + 4] and BF16 [128][BN + 8]
    static constexpr int kLdF = BN + 4, kLdH = BN + 8;
    static constexpr int kStageF = kBM * kLdF * 4, kStageH = kBM * kLdH * 2;
    static constexpr int kSmem = (kPipe > kStageF + kStageH ? kPipe : kStageF + kStageH) + 1024;
    // instruction descriptor: D FP32, A and B BF16, both K-major, M = 128, N = BN
    static constexpr uint32_t kIdesc =
        (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity)
{
    const uint32_t a = smem_u32(b);
    for (unsigned i = 0; i < kSpin; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)tm), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFF) | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}

template <int BN>
__global__ void __launch_bounds__(128, 2) k_gemm_tn(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB, const GemmEpi ep, int K,
                                                    int* err)
{
    using C = Cfg<BN>;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail, s_issued, s_consumed;
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
    const int KT = K / kBK;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        mbar_init(&done, 1);
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (tid == 0) {
        // producer: stage kt % kStages is refilled once the MMAs of step kt - kStages have completed
        for (int kt = 0; kt < KT; ++kt) {
            const int st = kt % kStages;
            if (kt >= kStages && !mbar_wait(&empty[st], (unsigned)(kt / kStages - 1) & 1u)) {
                s_fail = 1;
                break;
            }
            if (*(volatile int*)&s_fail) break;
            unsigned char* sa = smem + st * C::kStageBytes;
            mbar_expect_tx(&full[st], C::kStageBytes);
            tma_load_2d(sa, &tmA, kt * kBK, m0, &full[st]);
            tma_load_2d(sa + kTileA, &tmB, kt * kBK, n0, &full[st]);
            *(volatile int*)&s_issued = kt + 1;
        }
    } else if (tid == 32) {
        // MMA issuer
        bool ok = true;
        for (int kt = 0; kt < KT; ++kt) {
            const int st = kt % kStages;
            if (!mbar_wait(&full[st], (unsigned)(kt / kStages) & 1u)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + st * C::kStageBytes);
            const uint32_t sb = sa + kTileA;
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)
                mma_bf16(tmem, desc_sw128(sa + 32 * kk), desc_sw128(sb + 32 * kk), C::kIdesc, (kt | kk) != 0);
            mma_commit(&empty[st]);
            *(volatile int*)&s_consumed = kt + 1;
        }
        if (ok) mma_commit(&done);
        else *(volatile int*)&s_fail = 1;
    }
    // wait for the accumulator (or for the issuer to give up)
    bool ready = false;
    for (int r = 0; r < 4 && !ready; ++r) {
        ready = mbar_wait(&done, 0);
        if (*(volatile int*)&s_fail) break;
    }
    tc_fence_after();
    __syncthreads();  // all TMA writes and MMA reads of the pipeline buffers are over: reuse them
    if (!ready || s_fail) {
        if (tid == 0) {
            atomicExch(err, 1);
            // let the loads still in flight land before the CTA's shared memory goes away
            for (int kt = s_consumed; kt < s_issued; ++kt) mbar_wait(&full[kt % kStages], (unsigned)(kt / kStages) & 1u);
        }
    } else {
        float* sf = reinterpret_cast<float*>(smem);                          // FP32 [128][kLdF]
        __nv_bfloat16* sh = reinterpret_cast<__nv_bfloat16*>(smem + C::kStageF);  // BF16 [128][kLdH]
        const int r = warp * 32 + lane;  // tile row of this thread
        if (ep.mode == kEpiGeluGrad) {
            // stage the pre-activation tile with coalesced loads
            for (int q = tid; q < kBM * (BN / 4); q += 128) {
                const int rr = q / (BN / 4), cc = (q % (BN / 4)) * 4;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (m0 + rr < ep.M) v = *reinterpret_cast<const float4*>(ep.z + (size_t)(m0 + rr) * ep.ldz + n0 + cc);
                *reinterpret_cast<float4*>(sf + rr * C::kLdF + cc) = v;
            }
            __syncthreads();
        }
        for (int c0 = 0; c0 < BN; c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (ep.mode == kEpiF32) {
#pragma unroll
                for (int i = 0; i < 32; i += 4)
                    *reinterpret_cast<float4*>(sf + r * C::kLdF + c0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            } else if (ep.mode == kEpiBiasGelu) {
#pragma unroll
                for (int i = 0; i < 32; i += 2) {
                    const float z0 = v[i] + ep.bias[n0 + c0 + i], z1 = v[i + 1] + ep.bias[n0 + c0 + i + 1];
                    *reinterpret_cast<float2*>(sf + r * C::kLdF + c0 + i) = make_float2(z0, z1);
                    *reinterpret_cast<__nv_bfloat162*>(sh + r * C::kLdH + c0 + i) =
                        __floats2bfloat162_rn(gelu(z0), gelu(z1));
                }
            } else {  // kEpiGeluGrad: dz = acc * gelu'(z)
#pragma unroll
                for (int i = 0; i < 32; i += 2) {
                    const float2 z = *reinterpret_cast<const float2*>(sf + r * C::kLdF + c0 + i);
                    *reinterpret_cast<__nv_bfloat162*>(sh + r * C::kLdH + c0 + i) =
                        __floats2bfloat162_rn(v[i] * gelu_grad(z.x), v[i + 1] * gelu_grad(z.y));
                }
            }
        }
        __syncthreads();
        // coalesced write-out: consecutive threads take consecutive 16-byte pieces of a row
        if (ep.mode != kEpiGeluGrad) {
            for (int q = tid; q < kBM * (BN / 4); q += 128) {
                const int rr = q / (BN / 4), cc = (q % (BN / 4)) * 4;
                if (m0 + rr < ep.M)
                    *reinterpret_cast<float4*>(ep.c_f32 + (size_t)(m0 + rr) * ep.ldc + n0 + cc) =
                        *reinterpret_cast<const float4*>(sf + rr * C::kLdF + cc);
            }
        }
        if (ep.mode != kEpiF32) {
            for (int q = tid; q < kBM * (BN / 8); q += 128) {
                const int rr = q / (BN / 8), cc = (q % (BN / 8)) * 8;
                if (m0 + rr < ep.M)
                    *reinterpret_cast<uint4*>(ep.out_bf16 + (size_t)(m0 + rr) * ep.ldo + n0 + cc) =
                        *reinterpret_cast<const uint4*>(sh + rr * C::kLdH + cc);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t get_encode()
{
    if (g_encode) return cudaSuccess;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return cudaSuccess;
}

// 2-D BF16 tensor map over a row-major [rows x cols] matrix (row stride ld
// elements), box of 64 columns x box_rows rows, 128-byte swizzle
cudaError_t make_map(CUtensorMap* m, const void* base, int rows, int cols, int ld, int box_rows)
{
    cudaError_t e = get_encode();
    if (e != cudaSuccess) return e;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

bool gemm_shape_ok(int M, int N, int K)
{
    return M > 0 && N > 0 && K > 0 && M % kBM == 0 && N % 128 == 0 && K % kBK == 0;
}

namespace {

template <int BN>
cudaError_t launch_gemm(const void* A, int lda, const void* B, int ldb, int M, int N, int K, const GemmEpi& ep,
                        int* err, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_tn<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<BN>::kSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    CUtensorMap ta, tb;
    cudaError_t e = make_map(&ta, A, M, K, lda, kBM);
    if (e == cudaSuccess) e = make_map(&tb, B, N, K, ldb, BN);
    if (e != cudaSuccess) return e;
    dim3 grid(N / BN, M / kBM);
    k_gemm_tn<BN><<<grid, 128, Cfg<BN>::kSmem, st>>>(ta, tb, ep, K, err);
    return cudaGetLastError();
}

int g_sms = 0;

}  // namespace

// C = A B^T; A [M x K] (row stride lda), B [N x K] (row stride ldb), BF16, K-contiguous.
// 128 x 64 tiles when 128 x 128 tiles would cover fewer CTAs than SMs.
cudaError_t gemm_bf16_tn(const void* A, int lda, const void* B, int ldb, int M, int N, int K, const GemmEpi& ep,
                         int* err, cudaStream_t st)
{
    if (!gemm_shape_ok(M, N, K) || lda % 8 || ldb % 8 || ((uintptr_t)A & 15) || ((uintptr_t)B & 15))
        return cudaErrorInvalidValue;
    if (ep.mode != kEpiGeluGrad && (ep.ldc % 4 || ((uintptr_t)ep.c_f32 & 15))) return cudaErrorInvalidValue;
    if (ep.mode != kEpiF32 && (ep.ldo % 8 || ((uintptr_t)ep.out_bf16 & 15))) return cudaErrorInvalidValue;
    if (ep.mode == kEpiGeluGrad && (ep.ldz % 4 || ((uintptr_t)ep.z & 15))) return cudaErrorInvalidValue;
    if (!g_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    if ((long long)(M / kBM) * (N / 128) < g_sms) return launch_gemm<64>(A, lda, B, ldb, M, N, K, ep, err, st);
    return launch_gemm<128>(A, lda, B, ldb, M, N, K, ep, err, st);
}

}  // namespace sbr
