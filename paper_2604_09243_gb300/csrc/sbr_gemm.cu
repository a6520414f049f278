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
        if (ep.mode != kEpiGeluGrad && ep.c_f32) {
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

// ---------------------------------------------------------------- persistent form
// For grids of at least two 128 x 128 tiles per SM: one CTA per SM loops over
// the tiles t = blockIdx.x, t + gridDim.x, ... (n-tile fastest) with six warps.
// Warp 0 (one lane) streams the A and B tiles of every k-step of every tile
// through the 3-stage ring; warp 1 (one lane) issues the MMAs of the CTA's
// tile j into TMEM accumulator j % 2 (128 columns each) once the epilogue has
// drained it and commits it; warps 2-5 read their 32 rows of the accumulator
// (TMEM lanes 32 (w % 4) ..), release it, and apply the epilogue through
// staging rows of their own, so that a tile's read-out, epilogue and stores
// overlap the next tile's MMAs. The MMAs of a tile come in the same order and
// the epilogue does the same arithmetic as in k_gemm_tn: the results are the
// same bit for bit. Every wait is bounded and polls the CTA's failure flag.
constexpr int kPpStages = 3;
constexpr int kPpThreads = 192;
struct PpCfg {
    static constexpr int BN = 128;
    static constexpr int kStageBytes = kTileA + BN * kBK * 2;  // 32 KB
    static constexpr int kPipe = kPpStages * kStageBytes;
    static constexpr int kLdF = BN + 4, kLdH = BN + 8;
    static constexpr int kWarpF = 32 * kLdF * 4, kWarpH = 32 * kLdH * 2;  // staging of one epilogue warp
    static constexpr int kSmem = kPipe + 4 * (kWarpF + kWarpH) + 1024;
};
static_assert(PpCfg::kSmem <= 227 * 1024, "persistent GEMM shared memory");

// a bounded wait that also gives up once another role of the CTA has failed
__device__ __forceinline__ bool pp_wait(uint64_t* b, unsigned parity, volatile int* fail)
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
        if ((i & 1023u) == 1023u && *fail) return false;
    }
    return false;
}

__global__ void __launch_bounds__(kPpThreads, 1) k_gemm_pp(const __grid_constant__ CUtensorMap tmA,
                                                           const __grid_constant__ CUtensorMap tmB, const GemmEpi ep,
                                                           int K, int tiles_n, int n_tiles, int* err)
{
    using C = PpCfg;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kPpStages], empty[kPpStages], tfull[2], tempty[2], drained;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail, s_issued, s_consumed;
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int KT = K / kBK;
    const int my_tiles = (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    volatile int* fail = &s_fail;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int st = 0; st < kPpStages; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);  // one arrival per epilogue warp
        }
        mbar_init(&drained, 1);
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
        // producer: global k-step g of the CTA refills stage g % kPpStages once the MMAs of step g - kPpStages
        // have completed
        int g = 0;
        for (int j = 0; j < my_tiles && !*fail; ++j) {
            const int t = (int)blockIdx.x + j * (int)gridDim.x;
            const int m0 = (t / tiles_n) * kBM, n0 = (t % tiles_n) * C::BN;
            for (int kt = 0; kt < KT; ++kt, ++g) {
                const int st = g % kPpStages;
                if (g >= kPpStages && !pp_wait(&empty[st], (unsigned)(g / kPpStages - 1) & 1u, fail)) {
                    *fail = 1;
                    break;
                }
                unsigned char* sa = smem + st * C::kStageBytes;
                mbar_expect_tx(&full[st], C::kStageBytes);
                tma_load_2d(sa, &tmA, kt * kBK, m0, &full[st]);
                tma_load_2d(sa + kTileA, &tmB, kt * kBK, n0, &full[st]);
                *(volatile int*)&s_issued = g + 1;
            }
        }
    } else if (tid == 32) {
        // MMA issuer: tile j into accumulator j % 2 once the epilogue has drained tile j - 2 from it
        int g = 0;
        bool ok = true;
        for (int j = 0; j < my_tiles && ok; ++j) {
            const int b = j & 1;
            if (j >= 2 && !pp_wait(&tempty[b], (unsigned)((j >> 1) - 1) & 1u, fail)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t acc = tmem + (uint32_t)(b * C::BN);
            for (int kt = 0; kt < KT; ++kt, ++g) {
                const int st = g % kPpStages;
                if (!pp_wait(&full[st], (unsigned)(g / kPpStages) & 1u, fail)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + st * C::kStageBytes);
                const uint32_t sb = sa + kTileA;
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk)
                    mma_bf16(acc, desc_sw128(sa + 32 * kk), desc_sw128(sb + 32 * kk), Cfg<128>::kIdesc,
                             (kt | kk) != 0);
                mma_commit(&empty[st]);
                *(volatile int*)&s_consumed = g + 1;
            }
            if (ok) mma_commit(&tfull[b]);
        }
        if (!ok) *fail = 1;
        // every MMA issued has completed before the accumulators are freed (waited for even after a failure)
        mma_commit(&drained);
        mbar_wait(&drained, 0);
    } else if (warp >= 2) {
        // epilogue: warp w owns tile rows (TMEM lanes) 32 (w % 4) .. 32 (w % 4) + 31
        const int q = warp & 3;
        float* sf = reinterpret_cast<float*>(smem + C::kPipe + (warp - 2) * (C::kWarpF + C::kWarpH));
        __nv_bfloat16* sh = reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(sf) + C::kWarpF);
        for (int j = 0; j < my_tiles; ++j) {
            const int b = j & 1;
            const int t = (int)blockIdx.x + j * (int)gridDim.x;
            const int m0 = (t / tiles_n) * kBM + 32 * q, n0 = (t % tiles_n) * C::BN;
            // warp-uniform decision: the TMEM loads below are warp-collective
            if (!__all_sync(0xffffffffu, pp_wait(&tfull[b], (unsigned)(j >> 1) & 1u, fail))) {
                *fail = 1;
                break;
            }
            tc_fence_after();
            if (ep.mode == kEpiGeluGrad) {
                // the warp's 32 rows of the pre-activation, coalesced (lane l: columns 4 l .. 4 l + 3)
                for (int rr = 0; rr < 32; ++rr) {
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (m0 + rr < ep.M) v = *reinterpret_cast<const float4*>(ep.z + (size_t)(m0 + rr) * ep.ldz + n0 + 4 * lane);
                    *reinterpret_cast<float4*>(sf + rr * C::kLdF + 4 * lane) = v;
                }
                __syncwarp();
            }
            for (int c0 = 0; c0 < C::BN; c0 += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * C::BN + c0), v);
                if (ep.mode == kEpiF32) {
#pragma unroll
                    for (int i = 0; i < 32; i += 4)
                        *reinterpret_cast<float4*>(sf + lane * C::kLdF + c0 + i) =
                            make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                } else if (ep.mode == kEpiBiasGelu) {
#pragma unroll
                    for (int i = 0; i < 32; i += 2) {
                        const float z0 = v[i] + ep.bias[n0 + c0 + i], z1 = v[i + 1] + ep.bias[n0 + c0 + i + 1];
                        *reinterpret_cast<float2*>(sf + lane * C::kLdF + c0 + i) = make_float2(z0, z1);
                        *reinterpret_cast<__nv_bfloat162*>(sh + lane * C::kLdH + c0 + i) =
                            __floats2bfloat162_rn(gelu(z0), gelu(z1));
                    }
                } else {  // kEpiGeluGrad: dz = acc * gelu'(z)
#pragma unroll
                    for (int i = 0; i < 32; i += 2) {
                        const float2 z = *reinterpret_cast<const float2*>(sf + lane * C::kLdF + c0 + i);
                        *reinterpret_cast<__nv_bfloat162*>(sh + lane * C::kLdH + c0 + i) =
                            __floats2bfloat162_rn(v[i] * gelu_grad(z.x), v[i + 1] * gelu_grad(z.y));
                    }
                }
            }
            // the accumulator is in registers and staging: hand it back to the MMA issuer
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[b])) : "memory");
            if (ep.mode != kEpiGeluGrad && ep.c_f32)
                for (int rr = 0; rr < 32; ++rr)
                    if (m0 + rr < ep.M)
                        *reinterpret_cast<float4*>(ep.c_f32 + (size_t)(m0 + rr) * ep.ldc + n0 + 4 * lane) =
                            *reinterpret_cast<const float4*>(sf + rr * C::kLdF + 4 * lane);
            if (ep.mode != kEpiF32)
                for (int rr = 0; rr < 32; rr += 2) {
                    const int row = rr + (lane >> 4), col = 8 * (lane & 15);
                    if (m0 + row < ep.M)
                        *reinterpret_cast<uint4*>(ep.out_bf16 + (size_t)(m0 + row) * ep.ldo + n0 + col) =
                            *reinterpret_cast<const uint4*>(sh + row * C::kLdH + col);
                }
            __syncwarp();  // the staging rows are rewritten by the next tile
        }
    }
    tc_fence_before();
    __syncthreads();
    if (*fail && tid == 0) {
        atomicExch(err, 1);
        // let the loads still in flight land before the CTA's shared memory goes away
        for (int g = s_consumed; g < s_issued; ++g) mbar_wait(&full[g % kPpStages], (unsigned)(g / kPpStages) & 1u);
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
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
    if (ep.mode == kEpiF32 && !ep.c_f32) return cudaErrorInvalidValue;
    if (ep.mode != kEpiF32 && (ep.ldo % 8 || ((uintptr_t)ep.out_bf16 & 15))) return cudaErrorInvalidValue;
    if (ep.mode == kEpiGeluGrad && (ep.ldz % 4 || ((uintptr_t)ep.z & 15))) return cudaErrorInvalidValue;
    if (!g_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    const long long tiles = (long long)(M / kBM) * (N / 128);
    if (tiles < g_sms) return launch_gemm<64>(A, lda, B, ldb, M, N, K, ep, err, st);
    if (tiles >= 2ll * g_sms && tiles < (1ll << 31)) {
        // persistent: one CTA per SM, accumulators double-buffered in TMEM
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(k_gemm_pp, cudaFuncAttributeMaxDynamicSharedMemorySize, PpCfg::kSmem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        CUtensorMap ta, tb;
        cudaError_t e = make_map(&ta, A, M, K, lda, kBM);
        if (e == cudaSuccess) e = make_map(&tb, B, N, K, ldb, 128);
        if (e != cudaSuccess) return e;
        k_gemm_pp<<<g_sms, kPpThreads, PpCfg::kSmem, st>>>(ta, tb, ep, K, N / 128, (int)tiles, err);
        return cudaGetLastError();
    }
    return launch_gemm<128>(A, lda, B, ldb, M, N, K, ep, err, st);
}

}  // namespace sbr
