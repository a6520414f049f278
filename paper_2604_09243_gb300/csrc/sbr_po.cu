// sbr_po.cu -- physical-optics ray-tube sum over the dense valid-hit records
// (Eq. po_sum of the paper; vector form from Eq. em5/em6).
//
// The records of one aspect are cut into items of up to kPoItemRecords tubes. One
// block owns an item: it loads the tubes once and, for every requested
// frequency, evaluates e^{-j k L} per tube, multiplies by the tube coefficients
// and reduces with warp shuffles and a shared-memory tree in FP32. The item
// partial is stored in FP64; a second kernel adds the partials of an aspect in
// item order in FP64, applies -j k / (4 pi) and sigma = 4 pi |E|^2 (Sec. 4).
// The order of every addition is fixed, so results are bitwise reproducible
// (the paper notes run-to-run scatter of its FP32 sums, Sec. 5.1).
//
// Phase: k L is formed in cycles, kappa = f / c0, with kappa and L both held
// as unevaluated two-float sums; the integer part is dropped exactly and the
// fraction goes to sincospi. This keeps the phase error at the FP32 rounding
// of the fraction even for paths of thousands of wavelengths.
#include <math.h>

#include <algorithm>

#include "sbr_internal.h"

namespace sbr {

namespace {

constexpr int kPoThreads = 256;
constexpr int kWarps = kPoThreads / 32;

__device__ __forceinline__ void phase_cs(const PoArgs& a, float4 fq, double kd, float lh, float ll, float& c,
                                         float& s)
{
    if (a.phase_mode == 0) {
        const float p = __fmul_rn(fq.x, lh);
        float e = __fmaf_rn(fq.x, lh, -p);
        e = __fadd_rn(e, __fadd_rn(__fmul_rn(fq.x, ll), __fmul_rn(fq.y, lh)));
        const float n = rintf(p);
        const float r = __fadd_rn(__fsub_rn(p, n), e);
        sincospif(2.f * r, &s, &c);
    } else if (a.phase_mode == 1) {
        sincosf(fq.z * lh, &s, &c);
    } else {
        double sd, cd;
        sincos(kd * ((double)lh + (double)ll), &sd, &cd);
        s = (float)sd;
        c = (float)cd;
    }
}

// kPoPer records per thread: items of kPoPer * kPoThreads records
// kPoPer records per thread (items of kPoPer * kPoThreads records) and room for
// kPol polarisations (2 or 4). Every block reduction carries 8 sums: two
// frequencies at a time when kPol = 2, one when kPol = 4. Each sum is formed
// in the same order whatever kPol, so the results do not depend on it.
template <int kPoPer, int kPol>
__global__ void __launch_bounds__(kPoThreads) k_po(const PoArgs a)
{
    constexpr int kF = 4 / kPol;  // frequencies per block reduction
    __shared__ float s_red[kWarps][8];
    const int n_items = a.n_items_dev ? *a.n_items_dev : a.n_items;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const PoItem I = a.items[item];
        float cf[kPoPer][kPol];
        float lh[kPoPer], ll[kPoPer];
#pragma unroll
        for (int k = 0; k < kPoPer; ++k) {
            const int idx = k * kPoThreads + tid;
            if (idx < I.count) {
                const float4* p = reinterpret_cast<const float4*>(a.rec + I.first + idx);
                const float4 x = __ldg(p), y = __ldg(p + 1);
#pragma unroll
                for (int q = 0; q < kPol; ++q) {
                    // coefficient of polarisation pol_sel[q] (a selection, not an indexed local array)
                    const int sel = a.pol_sel[q];
                    const float vec = sel == 0 ? x.x : (sel == 1 ? x.y : (sel == 2 ? x.z : x.w));
                    float v = 0.f;
                    if (q < a.n_pol) v = a.scalar ? (sel < 2 ? y.x : 0.f) : vec;
                    cf[k][q] = v;
                }
                lh[k] = y.y;
                ll[k] = y.z;
            } else {
#pragma unroll
                for (int q = 0; q < kPol; ++q) cf[k][q] = 0.f;
                lh[k] = 0.f;
                ll[k] = 0.f;
            }
        }
        for (int f0 = 0; f0 < I.nf; f0 += kF) {
            float acc[8];
#pragma unroll
            for (int v = 0; v < 8; ++v) acc[v] = 0.f;
#pragma unroll
            for (int fj = 0; fj < kF; ++fj) {
                if (f0 + fj >= I.nf) break;
                const float4 fq = a.freq[I.f0 + f0 + fj];
                const double kd = a.kfreq[I.f0 + f0 + fj];
#pragma unroll
                for (int k = 0; k < kPoPer; ++k) {
                    if (k * kPoThreads + tid >= I.count) break;
                    float c, s;
                    phase_cs(a, fq, kd, lh[k], ll[k], c, s);
#pragma unroll
                    for (int q = 0; q < kPol; ++q) {
                        acc[(fj * kPol + q) * 2] = fmaf(cf[k][q], c, acc[(fj * kPol + q) * 2]);
                        acc[(fj * kPol + q) * 2 + 1] = fmaf(-cf[k][q], s, acc[(fj * kPol + q) * 2 + 1]);
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int v = 0; v < 8; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
            if (lane == 0)
#pragma unroll
                for (int v = 0; v < 8; ++v) s_red[w][v] = acc[v];
            __syncthreads();
            if (tid < 8) {
                const int fj = tid / (2 * kPol), r = tid - fj * (2 * kPol);  // r = 2 q + (0 re, 1 im)
                if (f0 + fj < I.nf && r < 2 * a.n_pol) {
                    float v = 0.f;
#pragma unroll
                    for (int k = 0; k < kWarps; ++k) v += s_red[k][tid];
                    a.partial[I.part + (size_t)(f0 + fj) * (2 * a.n_pol) + r] = (double)v;
                }
            }
            __syncthreads();
        }
    }
}

static_assert(kPoItemRecords == 4 * kPoThreads, "PO item size");

// ---------------------------------------------------------------- staged single-frequency sum
// With one frequency per block reduction (F <= 4 / kPol) the sum reads each
// 32-byte record once and is bound by memory. The records of the items a block
// owns are contiguous ranges; they are streamed in stages of kPoThreads records
// (8 KB) by cp.async.bulk into a ring of kBulkStages shared-memory buffers, one
// mbarrier each, issued ahead across item boundaries, so the loads of the next
// stages overlap the phases, sums and reductions of the current one. Thread t
// takes record k * kPoThreads + t of an item in stage k, in order, so every
// term and every addition is that of k_po: the sums are bit-identical.
constexpr int kBulkStages = 4;
constexpr unsigned kPoSpin = 1u << 22;  // try_wait rounds before a wait gives up

__device__ __forceinline__ uint32_t po_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool po_wait(uint64_t* bar, unsigned parity)
{
    const uint32_t b = po_smem(bar);
    for (unsigned i = 0; i < kPoSpin; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(b), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

template <int kPol>
__global__ void __launch_bounds__(kPoThreads) k_po_bulk(const PoArgs a)
{
    constexpr int kF = 4 / kPol;
    __shared__ __align__(128) float4 s_rec[kBulkStages][2 * kPoThreads];
    __shared__ __align__(8) uint64_t s_full[kBulkStages];
    __shared__ float s_red[kWarps][8];
    const int n_items = a.n_items_dev ? *a.n_items_dev : a.n_items;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < kBulkStages; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(po_smem(&s_full[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // producer (thread 0): the next stage to load, as (item, stage of the item), and the stages issued
    int p_item = blockIdx.x, p_k = 0;
    unsigned issued = 0;
    auto produce = [&]() {
        if (p_item >= n_items) return;
        const PoItem I = a.items[p_item];
        const int cnt = min(kPoThreads, I.count - p_k * kPoThreads);
        const int s = (int)(issued % kBulkStages);
        const unsigned bytes = (unsigned)cnt * (unsigned)sizeof(Record);
        // the block's reads of this buffer (generic proxy) come before the copy that overwrites it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(po_smem(&s_full[s])), "r"(bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                po_smem(&s_rec[s][0])),
            "l"(a.rec + I.first + (long long)p_k * kPoThreads), "r"(bytes), "r"(po_smem(&s_full[s]))
            : "memory");
        ++issued;
        if (++p_k * kPoThreads >= I.count) {
            p_k = 0;
            p_item += gridDim.x;
        }
    };
    if (tid == 0)
        for (int s = 0; s < kBulkStages; ++s) produce();
    unsigned used = 0;  // stages consumed
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const PoItem I = a.items[item];
        float acc[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[v] = 0.f;
        const int n_st = (I.count + kPoThreads - 1) / kPoThreads;
        for (int k = 0; k < n_st; ++k, ++used) {
            const int s = (int)(used % kBulkStages);
            const bool ok = po_wait(&s_full[s], (used / kBulkStages) & 1u);
            if (__syncthreads_or(!ok)) {
                // a stage did not arrive: flag it, poison this item's sums, and leave only once the copies
                // still in flight into this block's buffers have landed (each wait bounded again)
                if (tid == 0) {
                    atomicOr(a.err, 1);
                    for (int r = 0; r < I.nf * 2 * a.n_pol; ++r) a.partial[I.part + r] = __longlong_as_double(-1ll);
                    for (unsigned u = used; u < issued; ++u)
                        po_wait(&s_full[u % kBulkStages], (u / kBulkStages) & 1u);
                }
                return;
            }
            const int idx = k * kPoThreads + tid;
            const bool valid = idx < I.count;
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f), y = x;
            if (valid) {
                x = s_rec[s][2 * tid];
                y = s_rec[s][2 * tid + 1];
            }
            __syncthreads();  // every thread has read stage s: it can be refilled
            if (tid == 0) produce();
            if (!valid) continue;
            float cf[kPol];
#pragma unroll
            for (int q = 0; q < kPol; ++q) {
                const int sel = a.pol_sel[q];
                const float vec = sel == 0 ? x.x : (sel == 1 ? x.y : (sel == 2 ? x.z : x.w));
                float v = 0.f;
                if (q < a.n_pol) v = a.scalar ? (sel < 2 ? y.x : 0.f) : vec;
                cf[q] = v;
            }
#pragma unroll
            for (int fj = 0; fj < kF; ++fj) {
                if (fj >= I.nf) break;
                const float4 fq = a.freq[I.f0 + fj];
                const double kd = a.kfreq[I.f0 + fj];
                float c, sn;
                phase_cs(a, fq, kd, y.y, y.z, c, sn);
#pragma unroll
                for (int q = 0; q < kPol; ++q) {
                    acc[(fj * kPol + q) * 2] = fmaf(cf[q], c, acc[(fj * kPol + q) * 2]);
                    acc[(fj * kPol + q) * 2 + 1] = fmaf(-cf[q], sn, acc[(fj * kPol + q) * 2 + 1]);
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int v = 0; v < 8; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
        if (lane == 0)
#pragma unroll
            for (int v = 0; v < 8; ++v) s_red[w][v] = acc[v];
        __syncthreads();
        if (tid < 8) {
            const int fj = tid / (2 * kPol), r = tid - fj * (2 * kPol);
            if (fj < I.nf && r < 2 * a.n_pol) {
                float v = 0.f;
#pragma unroll
                for (int k = 0; k < kWarps; ++k) v += s_red[k][tid];
                a.partial[I.part + (size_t)fj * (2 * a.n_pol) + r] = (double)v;
            }
        }
        __syncthreads();
    }
}

// Work list, stage 1 (one block): 64-bit exclusive scans over the aspects of
// their item counts and partial sizes, in tiles of the block size.
__global__ void k_po_items_scan(const unsigned* recoff, PoAngle* angles, int na, int n_pol, int item_records,
                                int* n_items, long long* valid)
{
    __shared__ long long s_ni[32], s_np[32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    long long base_i = 0, base_p = 0;
    for (int t0 = 0; t0 < na; t0 += blockDim.x) {
        const int a = t0 + tid;
        long long ni = 0, np = 0;
        if (a < na) {
            const unsigned rc = recoff[a + 1] - recoff[a];
            ni = (rc + item_records - 1) / item_records;
            np = ni * (long long)angles[a].nf * 2 * n_pol;
        }
        // inclusive warp scans, then across warps
        long long xi = ni, xp = np;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long yi = __shfl_up_sync(0xffffffffu, xi, o), yp = __shfl_up_sync(0xffffffffu, xp, o);
            if (lane >= o) {
                xi += yi;
                xp += yp;
            }
        }
        if (lane == 31) {
            s_ni[w] = xi;
            s_np[w] = xp;
        }
        __syncthreads();
        long long wi = 0, wp = 0, ti = 0, tp = 0;
        for (int k = 0; k < nw; ++k) {
            if (k < w) {
                wi += s_ni[k];
                wp += s_np[k];
            }
            ti += s_ni[k];
            tp += s_np[k];
        }
        if (a < na) {
            PoAngle& A = angles[a];
            A.item_begin = (int)(base_i + wi + xi - ni);
            A.item_end = (int)(base_i + wi + xi);
            A.part = base_p + wp + xp - np;
        }
        base_i += ti;
        base_p += tp;
        __syncthreads();
    }
    if (tid == 0) {
        *n_items = (int)base_i;
        if (valid) *valid = recoff[na];
    }
}

// Work list, stage 2: one warp per aspect writes its items. recoff: the record
// offsets of the aspects (32-bit within a chunk, or 64-bit over a whole trace).
template <typename Off>
__global__ void k_po_items_fill(const Off* recoff, const PoAngle* angles, int na, int n_pol, int item_records,
                                PoItem* items)
{
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < na; a += nwarps) {
        const PoAngle A = angles[a];
        const long long r0 = (long long)recoff[a], rc = (long long)recoff[a + 1] - r0;
        for (int r = lane; r < A.item_end - A.item_begin; r += 32) {
            PoItem it;
            it.angle = a;
            it.count = (int)min((long long)item_records, rc - (long long)r * item_records);
            it.first = r0 + (long long)r * item_records;
            it.f0 = A.f0;
            it.nf = A.nf;
            it.part = A.part + (long long)r * A.nf * 2 * n_pol;
            items[A.item_begin + r] = it;
        }
    }
}

// one block per aspect; its threads stride over (frequency, polarisation) outputs
__global__ void k_po_final(const double* partial, const PoItem* items, const PoAngle* angles, const double* kfreq,
                           int n_pol, double* E, double* rcs)
{
    const PoAngle A = angles[blockIdx.x];
    for (int o = threadIdx.x; o < A.nf * n_pol; o += blockDim.x) {
        const int q = o / n_pol, p = o - q * n_pol;
        // item order, as written; the loads of 8 items are issued before their additions
        double sr = 0.0, si = 0.0;
        for (int it0 = A.item_begin; it0 < A.item_end; it0 += 8) {
            double vr[8], vi[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                vr[u] = 0.0;
                vi[u] = 0.0;
                if (it0 + u < A.item_end) {
                    const double* v = partial + items[it0 + u].part + (size_t)q * (2 * n_pol) + 2 * p;
                    vr[u] = v[0];
                    vi[u] = v[1];
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (it0 + u < A.item_end) {
                    sr += vr[u];
                    si += vi[u];
                }
        }
        // E = (-j k / 4 pi) (sr + j si)
        const double pre = kfreq[A.f0 + q] / (4.0 * 3.14159265358979323846);
        const double er = pre * si, ei = -pre * sr;
        const long long i = (A.out_row + q) * n_pol + p;
        if (E) {
            E[2 * i] = er;
            E[2 * i + 1] = ei;
        }
        if (rcs) rcs[i] = 10.0 * log10(4.0 * 3.14159265358979323846 * (er * er + ei * ei));
    }
}

}  // namespace

cudaError_t launch_po(const PoArgs& a, cudaStream_t st, int n_blocks)
{
    const int grid = n_blocks > 0 ? n_blocks : a.n_items;
    if (grid <= 0) return cudaSuccess;
    const int per = (a.item_records > 0 ? a.item_records : kPoItemRecords) / kPoThreads;
    const bool two = a.n_pol <= 2;
    if (a.err && n_blocks == 0 && a.n_freq <= (two ? 2 : 1) && (per == 2 || per == 4 || per == 8)) {
        // one block reduction per item: the staged kernel, one persistent wave
        int dev = 0, sms = 0, occ = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = two ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_po_bulk<2>, kPoThreads, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_po_bulk<4>, kPoThreads, 0);
        if (e != cudaSuccess) return e;
        const int g = (int)std::min<long long>(a.n_items, (long long)sms * std::max(occ, 1));
        if (two) k_po_bulk<2><<<g, kPoThreads, 0, st>>>(a);
        else k_po_bulk<4><<<g, kPoThreads, 0, st>>>(a);
        return cudaGetLastError();
    }
    if (per == 2) {
        if (two) k_po<2, 2><<<grid, kPoThreads, 0, st>>>(a);
        else k_po<2, 4><<<grid, kPoThreads, 0, st>>>(a);
    } else if (per == 8) {
        if (two) k_po<8, 2><<<grid, kPoThreads, 0, st>>>(a);
        else k_po<8, 4><<<grid, kPoThreads, 0, st>>>(a);
    } else if (per == 4) {
        if (two) k_po<4, 2><<<grid, kPoThreads, 0, st>>>(a);
        else k_po<4, 4><<<grid, kPoThreads, 0, st>>>(a);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_po_items(const unsigned* recoff, PoAngle* angles, int n_angles, int n_pol, int item_records,
                            PoItem* items, int* n_items, long long* valid, cudaStream_t st)
{
    if (n_angles <= 0 || item_records <= 0) return cudaErrorInvalidValue;
    k_po_items_scan<<<1, 1024, 0, st>>>(recoff, angles, n_angles, n_pol, item_records, n_items, valid);
    const int blocks = (int)std::min<long long>(((long long)n_angles * 32 + 255) / 256, 4096);
    k_po_items_fill<unsigned><<<blocks, 256, 0, st>>>(recoff, angles, n_angles, n_pol, item_records, items);
    return cudaGetLastError();
}

cudaError_t launch_po_items_fill(const long long* recoff, const PoAngle* angles, int n_angles, int n_pol,
                                 int item_records, PoItem* items, cudaStream_t st)
{
    if (n_angles <= 0 || item_records <= 0) return cudaErrorInvalidValue;
    const int blocks = (int)std::min<long long>(((long long)n_angles * 32 + 255) / 256, 4096);
    k_po_items_fill<long long><<<blocks, 256, 0, st>>>(recoff, angles, n_angles, n_pol, item_records, items);
    return cudaGetLastError();
}

cudaError_t launch_po_final(const double* partial, const PoItem* items, const PoAngle* angles, int n_angles,
                            const double* kfreq, int n_pol, double* E, double* rcs, cudaStream_t st)
{
    if (n_angles <= 0) return cudaSuccess;
    k_po_final<<<n_angles, 128, 0, st>>>(partial, items, angles, kfreq, n_pol, E, rcs);
    return cudaGetLastError();
}

}  // namespace sbr
