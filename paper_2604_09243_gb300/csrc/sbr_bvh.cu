// sbr_bvh.cu -- GPU LBVH builder.
//
// The paper builds its BVH on the host by recursive median or binned-SAH
// partitioning (Sec. 4, Algorithm 1). Here the whole build runs on the GPU:
//   1. triangle AABBs and centroids, scene boxes (ordered-integer atomics, exact)
//   2. 63-bit Morton codes of the centroids (21 bits per axis)
//   3. stable LSD radix sort of (code, triangle) pairs, 8 passes of 8 bits
//   4. Karras hierarchy: n - 1 internal nodes from the sorted codes, ties broken
//      by position (Karras 2012, "Maximizing parallelism in the construction of
//      BVHs, octrees and k-d trees")
//   5. bottom-up refit with one atomic arrival flag per node; the second arrival
//      unions the child boxes and evaluates the SAH cost of the paper,
//      C_T SA(P) + C(L) + C(R) against C_I N SA(P) for collapsing the subtree
//      into one leaf of at most leaf_max triangles
//   6. node emission (child boxes stored in the parent) and triangle reorder so
//      that every leaf is a contiguous range (Sec. 4: leaves reference
//      contiguous triangle ranges).
#include <float.h>

#include "sbr_internal.h"

namespace sbr {

namespace {

constexpr int kThreads = 256;
constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr int kRsWarps = kRsThreads / 32;

__device__ __forceinline__ unsigned f2o(float f)
{
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float o2f(unsigned u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

// acc layout (unsigned ordered floats): [0..2] vertex min, [3..5] vertex max,
// [6..8] centroid min, [9..11] centroid max
__global__ void k_acc_init(unsigned* acc, int* err)
{
    int t = threadIdx.x;
    if (t < 12) acc[t] = ((t % 6) < 3) ? 0xFFFFFFFFu : 0u;
    if (t == 0) *err = 0;
}

__device__ __forceinline__ void warp_minmax_atomic(float3 lo, float3 hi, unsigned* acc_lo, unsigned* acc_hi)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
        lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
        lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o));
        hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
        hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
        hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (lo.x <= hi.x) {
            atomicMin(acc_lo + 0, f2o(lo.x));
            atomicMin(acc_lo + 1, f2o(lo.y));
            atomicMin(acc_lo + 2, f2o(lo.z));
            atomicMax(acc_hi + 0, f2o(hi.x));
            atomicMax(acc_hi + 1, f2o(hi.y));
            atomicMax(acc_hi + 2, f2o(hi.z));
        }
    }
}

// err bit 1: a triangle index out of range; bit 2: a non-finite vertex coordinate
__global__ void __launch_bounds__(kThreads) k_vertex_box(const float* xyz, long long nv, unsigned* acc, int* err)
{
    float3 lo = make_float3(FLT_MAX, FLT_MAX, FLT_MAX), hi = make_float3(-FLT_MAX, -FLT_MAX, -FLT_MAX);
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
        float x = xyz[3 * v], y = xyz[3 * v + 1], z = xyz[3 * v + 2];
        if (!isfinite(x) || !isfinite(y) || !isfinite(z)) atomicOr(err, 2);
        lo = make_float3(fminf(lo.x, x), fminf(lo.y, y), fminf(lo.z, z));
        hi = make_float3(fmaxf(hi.x, x), fmaxf(hi.y, y), fmaxf(hi.z, z));
    }
    warp_minmax_atomic(lo, hi, acc, acc + 3);
}

__global__ void __launch_bounds__(kThreads) k_prep(const float* xyz, const int* tri, long long nv, int n,
                                                   float4* tbox, float4* cen, unsigned* acc, int* err)
{
    float3 lo = make_float3(FLT_MAX, FLT_MAX, FLT_MAX), hi = make_float3(-FLT_MAX, -FLT_MAX, -FLT_MAX);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int ia = tri[3 * (long long)i], ib = tri[3 * (long long)i + 1], ic = tri[3 * (long long)i + 2];
        const bool bad = ia < 0 || ib < 0 || ic < 0 || ia >= nv || ib >= nv || ic >= nv;
        if (bad) {
            atomicOr(err, 1);
            ia = ib = ic = 0;
        }
        float3 a = make_float3(xyz[3 * (long long)ia], xyz[3 * (long long)ia + 1], xyz[3 * (long long)ia + 2]);
        float3 b = make_float3(xyz[3 * (long long)ib], xyz[3 * (long long)ib + 1], xyz[3 * (long long)ib + 2]);
        float3 c = make_float3(xyz[3 * (long long)ic], xyz[3 * (long long)ic + 1], xyz[3 * (long long)ic + 2]);
        // a refused mesh (bad index, non-finite vertex: flagged above and in
        // k_vertex_box) still completes its build with finite boxes
        if (bad || !isfinite(a.x + a.y + a.z + b.x + b.y + b.z + c.x + c.y + c.z))
            a = b = c = make_float3(0.f, 0.f, 0.f);
        float3 bl = make_float3(fminf(a.x, fminf(b.x, c.x)), fminf(a.y, fminf(b.y, c.y)), fminf(a.z, fminf(b.z, c.z)));
        float3 bh = make_float3(fmaxf(a.x, fmaxf(b.x, c.x)), fmaxf(a.y, fmaxf(b.y, c.y)), fmaxf(a.z, fmaxf(b.z, c.z)));
        // widen the leaf box well beyond the FP32 slab test's rounding (a few
        // units of the coordinates' magnitude) so that no box of a triangle the
        // exact test accepts is culled
        const float ext = fmaxf(bh.x - bl.x, fmaxf(bh.y - bl.y, bh.z - bl.z));
        const float mag = fmaxf(fmaxf(fmaxf(fabsf(bl.x), fabsf(bh.x)), fmaxf(fabsf(bl.y), fabsf(bh.y))),
                                fmaxf(fabsf(bl.z), fabsf(bh.z)));
        const float grow = ext * 0x1p-11f + mag * 0x1p-19f + 1e-30f;
        tbox[2 * i] = make_float4(bl.x - grow, bl.y - grow, bl.z - grow, 0.f);
        tbox[2 * i + 1] = make_float4(bh.x + grow, bh.y + grow, bh.z + grow, 0.f);
        float3 m = make_float3((a.x + b.x + c.x) * (1.f / 3.f), (a.y + b.y + c.y) * (1.f / 3.f),
                               (a.z + b.z + c.z) * (1.f / 3.f));
        cen[i] = make_float4(m.x, m.y, m.z, 0.f);
        lo = make_float3(fminf(lo.x, m.x), fminf(lo.y, m.y), fminf(lo.z, m.z));
        hi = make_float3(fmaxf(hi.x, m.x), fmaxf(hi.y, m.y), fmaxf(hi.z, m.z));
    }
    warp_minmax_atomic(lo, hi, acc + 6, acc + 9);
}

__device__ __forceinline__ unsigned long long spread21(unsigned long long x)
{
    x &= 0x1fffffull;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__global__ void __launch_bounds__(kThreads) k_morton(const float4* cen, int n, const unsigned* acc,
                                                     unsigned long long* keys, unsigned* vals, float* bbox_out)
{
    float lo[3], sc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lo[c] = o2f(acc[6 + c]);
        float ext = o2f(acc[9 + c]) - lo[c];
        sc[c] = ext > 0.f ? 2097152.f / ext : 0.f;
    }
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && bbox_out)
        for (int c = 0; c < 6; ++c) bbox_out[c] = o2f(acc[c]);
    if (i >= n) return;
    float4 m = cen[i];
    unsigned q[3];
    float mc[3] = {m.x, m.y, m.z};
#pragma unroll
    for (int c = 0; c < 3; ++c) q[c] = (unsigned)fminf(fmaxf((mc[c] - lo[c]) * sc[c], 0.f), 2097151.f);
    keys[i] = (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);
    vals[i] = (unsigned)i;
}

// ---------------------------------------------------------------- radix sort
__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const unsigned long long* keys, int n, int shift,
                                                        unsigned* hist, int nb)
{
    __shared__ unsigned s_h[256];
    s_h[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * kRsTile;
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) {
        int i = base + r * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&s_h[(unsigned)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * nb + blockIdx.x] = s_h[threadIdx.x];  // digit-major
}

// stable scatter: keys of a tile are ranked in index order, warp by warp
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const unsigned long long* kin, const unsigned* vin,
                                                           unsigned long long* kout, unsigned* vout, int n,
                                                           int shift, const unsigned* hist, int nb)
{
    __shared__ unsigned s_base[256];
    __shared__ unsigned s_cnt[kRsWarps][256];
    __shared__ unsigned s_off[kRsWarps][256];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    s_base[t] = hist[t * nb + blockIdx.x];
#pragma unroll
    for (int k = 0; k < kRsWarps; ++k) s_cnt[k][t] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    int base = blockIdx.x * kRsTile;
    for (int r = 0; r < kRsItems; ++r) {
        int i = base + r * kRsThreads + t;
        bool ok = i < n;
        unsigned long long key = ok ? kin[i] : 0ull;
        unsigned val = ok ? vin[i] : 0u;
        unsigned d = ok ? ((unsigned)(key >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned rank = __popc(peers & lt);
        if (ok && rank == 0) s_cnt[w][d] = __popc(peers);
        __syncthreads();
        {
            unsigned run = s_base[t];
#pragma unroll
            for (int k = 0; k < kRsWarps; ++k) {
                s_off[k][t] = run;
                run += s_cnt[k][t];
                s_cnt[k][t] = 0;
            }
            s_base[t] = run;
        }
        __syncthreads();
        if (ok) {
            unsigned dst = s_off[w][d] + rank;
            if (dst < (unsigned)n) {
                kout[dst] = key;
                vout[dst] = val;
            }
        }
    }
}

// ---------------------------------------------------------------- Karras hierarchy
__device__ __forceinline__ int delta(const unsigned long long* k, int n, int i, int j)
{
    if (j < 0 || j >= n) return -1;
    unsigned long long a = k[i], b = k[j];
    if (a == b) return 64 + __clz((unsigned)(i ^ j));
    return __clzll(a ^ b);
}

// child encoding: c >= 0 internal node c, c < 0 leaf ~c (sorted primitive)
__global__ void __launch_bounds__(kThreads) k_karras(const unsigned long long* k, int n, int* left, int* right,
                                                     int* first, int* last, int* par_int, int* par_leaf)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(k, n, i, i - d);
    int lmax = 2;
    while (delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta(k, n, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(k, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int g = i + s * d + min(d, 0);
    int lo = min(i, j), hi = max(i, j);
    int lc = (lo == g) ? ~g : g;
    int rc = (hi == g + 1) ? ~(g + 1) : g + 1;
    left[i] = lc;
    right[i] = rc;
    first[i] = lo;
    last[i] = hi;
    if (lc >= 0) par_int[lc] = i; else par_leaf[~lc] = i;
    if (rc >= 0) par_int[rc] = i; else par_leaf[~rc] = i;
}

__device__ __forceinline__ float area(float4 lo, float4 hi)
{
    float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return 2.f * (dx * dy + dy * dz + dz * dx);
}

// bottom-up refit; leaf data: lbox (sorted order); node data: nbox, ncnt, ncost, ncol
__global__ void __launch_bounds__(kThreads) k_refit(const unsigned* vals, const float4* tbox, int n,
                                                    const int* left, const int* right, const int* par_int,
                                                    const int* par_leaf, int* flags, float4* lbox, float4* nbox,
                                                    int* ncnt, float* ncost, int* ncol, int leaf_max, float c_t,
                                                    float c_i)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    unsigned tid = vals[p];
    lbox[2 * p] = tbox[2 * tid];
    lbox[2 * p + 1] = tbox[2 * tid + 1];
    if (n == 1) return;
    __threadfence();
    int node = par_leaf[p];
    // a walk to the root passes at most n - 1 internal nodes; the bound guards
    // against a malformed hierarchy
    for (int steps = 0; steps < n && node >= 0 && node < n - 1; ++steps) {
        if (atomicAdd(&flags[node], 1) == 0) return;  // first arrival: the sibling finishes the node
        __threadfence();
        int ch[2] = {left[node], right[node]};
        float4 lo = make_float4(FLT_MAX, FLT_MAX, FLT_MAX, 0.f), hi = make_float4(-FLT_MAX, -FLT_MAX, -FLT_MAX, 0.f);
        int cnt = 0;
        float cost = 0.f;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            float4 a, b;
            int c = ch[s];
            if (c < 0) {
                a = __ldcg(lbox + 2 * (~c));
                b = __ldcg(lbox + 2 * (~c) + 1);
                cnt += 1;
                cost += c_i * area(a, b);
            } else {
                a = __ldcg(nbox + 2 * c);
                b = __ldcg(nbox + 2 * c + 1);
                cnt += __ldcg(ncnt + c);
                cost += __ldcg(ncost + c);
            }
            lo = make_float4(fminf(lo.x, a.x), fminf(lo.y, a.y), fminf(lo.z, a.z), 0.f);
            hi = make_float4(fmaxf(hi.x, b.x), fmaxf(hi.y, b.y), fmaxf(hi.z, b.z), 0.f);
        }
        float sa = area(lo, hi);
        float split = c_t * sa + cost;
        float as_leaf = c_i * (float)cnt * sa;
        int col = (cnt <= leaf_max) && (as_leaf <= split);
        nbox[2 * node] = lo;
        nbox[2 * node + 1] = hi;
        ncnt[node] = cnt;
        ncost[node] = col ? as_leaf : split;
        ncol[node] = col;
        __threadfence();
        if (node == 0) return;
        node = par_int[node];
    }
}


__device__ __forceinline__ void put_node(float4* out, int i, float4 llo, float4 lhi, float4 rlo, float4 rhi, int lr,
                                         int rr)
{
    out[4 * i + 0] = make_float4(llo.x, lhi.x, llo.y, lhi.y);
    out[4 * i + 1] = make_float4(rlo.x, rhi.x, rlo.y, rhi.y);
    out[4 * i + 2] = make_float4(llo.z, lhi.z, rlo.z, rhi.z);
    out[4 * i + 3] = make_float4(__int_as_float(lr), __int_as_float(rr), 0.f, 0.f);
}

__global__ void __launch_bounds__(kThreads) k_emit(int n, const int* left, const int* right, const int* first,
                                                   const float4* lbox, const float4* nbox, const int* ncnt,
                                                   const int* ncol, float4* nodes)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float4 elo = make_float4(FLT_MAX, FLT_MAX, FLT_MAX, 0.f), ehi = make_float4(-FLT_MAX, -FLT_MAX, -FLT_MAX, 0.f);
    if (n == 1) {
        if (i == 0) put_node(nodes, 0, lbox[0], lbox[1], elo, ehi, leaf_ref(0, 1), kEmptyRef);
        return;
    }
    if (i >= n - 1) return;
    if (i == 0 && ncol[0]) {
        put_node(nodes, 0, nbox[0], nbox[1], elo, ehi, leaf_ref(0, ncnt[0]), kEmptyRef);
        return;
    }
    // every slot is written, those of collapsed clusters too (never reached from the root; their children
    // lie inside them), so that no slot keeps a node of an earlier build
    float4 bl[2], bh[2];
    int ref[2];
    int ch[2] = {left[i], right[i]};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        int c = ch[s];
        if (c < 0) {
            bl[s] = lbox[2 * (~c)];
            bh[s] = lbox[2 * (~c) + 1];
            ref[s] = leaf_ref(~c, 1);
        } else {
            bl[s] = nbox[2 * c];
            bh[s] = nbox[2 * c + 1];
            ref[s] = ncol[c] ? leaf_ref(first[c], ncnt[c]) : c;
        }
    }
    put_node(nodes, i, bl[0], bh[0], bl[1], bh[1], ref[0], ref[1]);
}

// FP64 vectors of the per-triangle preprocessing, each operation one IEEE
// rounding (no contraction): the unit normal and the degeneracy test below are
// the same FP64 evaluations as the oracle's, so both keep the same FP32 normal.
struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 dcross(D3 a, D3 b)
{
    return {__dsub_rn(__dmul_rn(a.y, b.z), __dmul_rn(a.z, b.y)), __dsub_rn(__dmul_rn(a.z, b.x), __dmul_rn(a.x, b.z)),
            __dsub_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x))};
}
__device__ __forceinline__ double ddot(D3 a, D3 b)
{
    return __dadd_rn(__dadd_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)), __dmul_rn(a.z, b.z));
}

__global__ void __launch_bounds__(kThreads) k_reorder(const float* xyz, const int* tri, long long nv,
                                                      const unsigned* vals, int n, float4* tris, float4* nrm,
                                                      float4* v12, int* pos)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    unsigned t = vals[p];
    int ia = tri[3 * (long long)t], ib = tri[3 * (long long)t + 1], ic = tri[3 * (long long)t + 2];
    if (ia < 0 || ib < 0 || ic < 0 || ia >= nv || ib >= nv || ic >= nv) ia = ib = ic = 0;
    float ax = xyz[3 * (long long)ia], ay = xyz[3 * (long long)ia + 1], az = xyz[3 * (long long)ia + 2];
    float bx = xyz[3 * (long long)ib], by = xyz[3 * (long long)ib + 1], bz = xyz[3 * (long long)ib + 2];
    float cx = xyz[3 * (long long)ic], cy = xyz[3 * (long long)ic + 1], cz = xyz[3 * (long long)ic + 2];
    float4 e1 = make_float4(__fsub_rn(bx, ax), __fsub_rn(by, ay), __fsub_rn(bz, az), 0.f);
    float4 e2 = make_float4(__fsub_rn(cx, ax), __fsub_rn(cy, ay), __fsub_rn(cz, az), 0.f);
    // Exact edges (differences of FP32 values) and the normal N = E1 x E2 in FP64.
    // Degenerate triangle: |N|^2 <= (2^-20 |E1|^2)(2^-20 |E2|^2), i.e. the sine of
    // the angle between its edges is at most 2^-20 (repeated or collinear vertices
    // give 0): it has no usable normal and takes no hits. Its edges and filter
    // constants are zeroed, which makes the test reject every ray.
    const D3 E1 = {__dsub_rn(bx, ax), __dsub_rn(by, ay), __dsub_rn(bz, az)};
    const D3 E2 = {__dsub_rn(cx, ax), __dsub_rn(cy, ay), __dsub_rn(cz, az)};
    const D3 N = dcross(E1, E2);
    const double nn = ddot(N, N), l1 = ddot(E1, E1), l2 = ddot(E2, E2);
    const bool deg = nn <= __dmul_rn(__dmul_rn(l1, 0x1p-20), __dmul_rn(l2, 0x1p-20));
    float4 n32 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (deg) {
        e1 = e2 = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        const double ln = __dsqrt_rn(nn);
        n32 = make_float4(__double2float_rn(__ddiv_rn(N.x, ln)), __double2float_rn(__ddiv_rn(N.y, ln)),
                          __double2float_rn(__ddiv_rn(N.z, ln)), 0.f);
        // filter constants of the FP32 test's forward error bounds (u = 2^-24)
        const float L = fmaxf(fabsf(e1.x) + fabsf(e1.y) + fabsf(e1.z), fabsf(e2.x) + fabsf(e2.y) + fabsf(e2.z));
        e1.w = (24.f * 0x1p-24f * 1.0009765625f) * L;
        e2.w = (14.f * 0x1p-24f * 1.0009765625f) * L * L;
    }
    tris[3 * p + 0] = make_float4(ax, ay, az, __int_as_float((int)t));
    tris[3 * p + 1] = e1;
    tris[3 * p + 2] = e2;
    nrm[p] = n32;
    v12[2 * p] = make_float4(bx, by, bz, 0.f);
    v12[2 * p + 1] = make_float4(cx, cy, cz, 0.f);
    if (pos) pos[t] = p;
}

// ---------------------------------------------------------------- PLOC builder
// Agglomerative clustering over the Morton-ordered triangles: every round,
// each cluster looks for the cluster within `radius` positions whose union
// box has the smallest surface area (ties: the lower position); mutual nearest
// neighbours merge into a new node, the survivors are compacted, until one
// cluster is left. Node ids count down from n - 2, so the root is node 0 and
// a node's id is below its children's. The SAH leaf-collapse decision of each
// node is taken when it is made, from its children's costs (same rule as the
// LBVH refit). A top-down pass then gives every node the first position of
// its triangles, so each collapsed subtree is a contiguous range.
struct Clusters {
    float4* lo;
    float4* hi;
    int* ref;    // >= 0 node id, < 0 ~triangle id
    int* cnt;
    float* cost;
};

__device__ __forceinline__ void ploc_init_one(int i, const unsigned* vals, const float4* tbox, float c_i, Clusters c)
{
    const unsigned t = vals[i];
    const float4 lo = tbox[2 * (size_t)t], hi = tbox[2 * (size_t)t + 1];
    c.lo[i] = lo;
    c.hi[i] = hi;
    c.ref[i] = ~(int)t;
    c.cnt[i] = 1;
    c.cost[i] = c_i * area(lo, hi);
}

__global__ void __launch_bounds__(kThreads) k_ploc_init(const unsigned* vals, const float4* tbox, int n, float c_i,
                                                        Clusters c)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) ploc_init_one(i, vals, tbox, c_i, c);
}

__device__ __forceinline__ float union_area(float4 al, float4 ah, float4 bl, float4 bh)
{
    return area(make_float4(fminf(al.x, bl.x), fminf(al.y, bl.y), fminf(al.z, bl.z), 0.f),
                make_float4(fmaxf(ah.x, bh.x), fmaxf(ah.y, bh.y), fmaxf(ah.z, bh.z), 0.f));
}

__device__ __forceinline__ void ploc_nn_one(int i, int m, int radius, Clusters c, int* nn)
{
    const float4 lo = c.lo[i], hi = c.hi[i];
    float best = FLT_MAX;
    int bj = -1;
    const int j0 = max(0, i - radius), j1 = min(m - 1, i + radius);
    for (int j = j0; j <= j1; ++j) {
        if (j == i) continue;
        const float a = union_area(lo, hi, c.lo[j], c.hi[j]);
        if (a < best) {  // strict: the lowest position wins ties
            best = a;
            bj = j;
        }
    }
    nn[i] = bj;
}

__global__ void __launch_bounds__(kThreads) k_ploc_nn(const int* m_dev, int radius, Clusters c, int* nn)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = *m_dev;
    if (i < m) ploc_nn_one(i, m, radius, c, nn);
}

// par / rel: parent and offset within the parent of node x (x < n - 1) or of
// triangle t (x = n - 1 + t), for the pointer-jumping position pass
// node arrays written by the merges
struct PlocNodes {
    int* left;
    int* right;
    float4* nbox;
    int* ncnt;
    float* ncost;
    int* ncol;
    int* par;  // parent and offset within the parent of node x or triangle n - 1 + t
    int* rel;
};

// cluster i < m of this round: merge with its mutual nearest neighbour
__device__ __forceinline__ void ploc_merge_one(int i, int n, Clusters c, const int* nn, int* next_id, PlocNodes g,
                                               unsigned* keep, int leaf_max, float c_t, float c_i)
{
    int* left = g.left;
    int* right = g.right;
    float4* nbox = g.nbox;
    int* ncnt = g.ncnt;
    float* ncost = g.ncost;
    int* ncol = g.ncol;
    int* par = g.par;
    int* rel = g.rel;
    const int j = nn[i];
    if (j < 0 || nn[j] != i) {
        keep[i] = 1;  // no mutual partner this round
        return;
    }
    if (i > j) {
        keep[i] = 0;  // merged into j
        return;
    }
    const float4 al = c.lo[i], ah = c.hi[i], bl = c.lo[j], bh = c.hi[j];
    const float4 lo = make_float4(fminf(al.x, bl.x), fminf(al.y, bl.y), fminf(al.z, bl.z), 0.f);
    const float4 hi = make_float4(fmaxf(ah.x, bh.x), fmaxf(ah.y, bh.y), fmaxf(ah.z, bh.z), 0.f);
    const int cnt = c.cnt[i] + c.cnt[j];
    const float sa = area(lo, hi);
    const float split = c_t * sa + c.cost[i] + c.cost[j];
    const float as_leaf = c_i * (float)cnt * sa;
    const int col = (cnt <= leaf_max) && (as_leaf <= split);
    const int id = atomicSub(next_id, 1);
    const int ri = c.ref[i], rj = c.ref[j];
    left[id] = ri;
    right[id] = rj;
    const int xi = ri >= 0 ? ri : n - 1 + ~ri, xj = rj >= 0 ? rj : n - 1 + ~rj;
    par[xi] = id;
    rel[xi] = 0;
    par[xj] = id;
    rel[xj] = c.cnt[i];
    nbox[2 * id] = lo;
    nbox[2 * id + 1] = hi;
    ncnt[id] = cnt;
    ncost[id] = col ? as_leaf : split;
    ncol[id] = col;
    c.lo[i] = lo;
    c.hi[i] = hi;
    c.ref[i] = id;
    c.cnt[i] = cnt;
    c.cost[i] = col ? as_leaf : split;
    keep[i] = 1;
}

__global__ void __launch_bounds__(kThreads) k_ploc_merge(const int* m_dev, int m_ub, int n, Clusters c, const int* nn,
                                                         int* next_id, PlocNodes g, unsigned* keep, int leaf_max,
                                                         float c_t, float c_i)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m_ub) return;
    if (i >= *m_dev) {
        keep[i] = 0;  // beyond the live clusters of this round
        return;
    }
    ploc_merge_one(i, n, c, nn, next_id, g, keep, leaf_max, c_t, c_i);
}

__device__ __forceinline__ void ploc_compact_one(int i, Clusters in, const unsigned* keep, const unsigned* pos,
                                                 Clusters out)
{
    if (!keep[i]) return;
    const unsigned k = pos[i];
    out.lo[k] = in.lo[i];
    out.hi[k] = in.hi[i];
    out.ref[k] = in.ref[i];
    out.cnt[k] = in.cnt[i];
    out.cost[k] = in.cost[i];
}

__global__ void __launch_bounds__(kThreads) k_ploc_compact(int m_ub, Clusters in, const unsigned* keep,
                                                           const unsigned* pos, Clusters out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m_ub) ploc_compact_one(i, in, keep, pos, out);
}

// position pass by pointer jumping: after round r every entry holds the sum of
// rel over its nearest 2^r ancestors and points 2^r levels up; once every
// pointer has left the root, rel is the first position of the node's triangles
__device__ __forceinline__ void ploc_jump_one(int x, const int* par_in, const int* rel_in, int* par_out, int* rel_out)
{
    const int p = par_in[x];
    if (p < 0) {
        par_out[x] = p;
        rel_out[x] = rel_in[x];
    } else {
        par_out[x] = par_in[p];
        rel_out[x] = rel_in[x] + rel_in[p];
    }
}

__global__ void __launch_bounds__(kThreads) k_ploc_jump(int count, const int* par_in, const int* rel_in, int* par_out,
                                                        int* rel_out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < count) ploc_jump_one(x, par_in, rel_in, par_out, rel_out);
}

__device__ __forceinline__ void ploc_positions_one(int x, int n, const int* rel, int* noff, unsigned* perm)
{
    if (x < n - 1) noff[x] = rel[x];
    else if (x < 2 * n - 1) perm[rel[x]] = (unsigned)(x - (n - 1));
}

__global__ void __launch_bounds__(kThreads) k_ploc_positions(int n, const int* rel, int* noff, unsigned* perm)
{
    ploc_positions_one(blockIdx.x * blockDim.x + threadIdx.x, n, rel, noff, perm);
}

__global__ void __launch_bounds__(kThreads) k_ploc_emit(int n, const int* left, const int* right, const float4* nbox,
                                                        const int* ncnt, const int* ncol, const int* noff,
                                                        const float4* tbox, float4* nodes)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const float4 elo = make_float4(FLT_MAX, FLT_MAX, FLT_MAX, 0.f), ehi = make_float4(-FLT_MAX, -FLT_MAX, -FLT_MAX, 0.f);
    if (i == 0 && ncol[0]) {
        put_node(nodes, 0, nbox[0], nbox[1], elo, ehi, leaf_ref(0, ncnt[0]), kEmptyRef);
        return;
    }
    float4 bl[2], bh[2];
    int ref[2];
    const int ch[2] = {left[i], right[i]};
    int off = noff[i];
    for (int s = 0; s < 2; ++s) {
        const int c = ch[s];
        if (c < 0) {
            bl[s] = tbox[2 * (size_t)(~c)];
            bh[s] = tbox[2 * (size_t)(~c) + 1];
            ref[s] = leaf_ref(off, 1);
            off += 1;
        } else {
            bl[s] = nbox[2 * c];
            bh[s] = nbox[2 * c + 1];
            ref[s] = ncol[c] ? leaf_ref(off, ncnt[c]) : c;
            off += ncnt[c];
        }
    }
    put_node(nodes, i, bl[0], bh[0], bl[1], bh[1], ref[0], ref[1]);
}

// ---------------------------------------------------------------- 4-wide collapse
__device__ __forceinline__ float half_area(float4 lo, float4 hi)
{
    const float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return dx * dy + dy * dz + dz * dx;
}

// children (box, ref) of binary node b; a missing child has ref kEmptyRef
__device__ __forceinline__ void binary_children(const float4* nodes2, int b, float4* lo, float4* hi, int* ref)
{
    const float4 n0 = nodes2[4 * (size_t)b], n1 = nodes2[4 * (size_t)b + 1], n2 = nodes2[4 * (size_t)b + 2],
                 n3 = nodes2[4 * (size_t)b + 3];
    lo[0] = make_float4(n0.x, n0.z, n2.x, 0.f);
    hi[0] = make_float4(n0.y, n0.w, n2.y, 0.f);
    lo[1] = make_float4(n1.x, n1.z, n2.z, 0.f);
    hi[1] = make_float4(n1.y, n1.w, n2.w, 0.f);
    ref[0] = __float_as_int(n3.x);
    ref[1] = __float_as_int(n3.y);
}

// One level: every queued (binary node, 4-wide slot) pair opens binary
// children, largest surface area first, until it has 4 children or only
// leaves; its internal children get new slots and go to the next level's queue.
__device__ __forceinline__ void collapse4_one(const float4* nodes2, int2 job, int2* qout, int* nout, int* count4,
                                              float4* nodes4)
{
    float4 lo[4], hi[4];
    int ref[4];
    int cnt = 0;
    {
        float4 l2[2], h2[2];
        int r2[2];
        binary_children(nodes2, job.x, l2, h2, r2);
        for (int c = 0; c < 2; ++c)
            if (r2[c] != kEmptyRef) {
                lo[cnt] = l2[c];
                hi[cnt] = h2[c];
                ref[cnt] = r2[c];
                ++cnt;
            }
    }
    while (cnt < 4) {
        int best = -1;
        float ba = -1.f;
        for (int c = 0; c < cnt; ++c)
            if (ref[c] >= 0) {
                const float a = half_area(lo[c], hi[c]);
                if (a > ba) {
                    ba = a;
                    best = c;
                }
            }
        if (best < 0) break;
        float4 l2[2], h2[2];
        int r2[2];
        binary_children(nodes2, ref[best], l2, h2, r2);
        lo[best] = l2[0];
        hi[best] = h2[0];
        ref[best] = r2[0];
        if (r2[1] != kEmptyRef) {
            lo[cnt] = l2[1];
            hi[cnt] = h2[1];
            ref[cnt] = r2[1];
            ++cnt;
        }
    }
    for (int c = 0; c < cnt; ++c)
        if (ref[c] >= 0) {
            const int t = atomicAdd(count4, 1);
            qout[atomicAdd(nout, 1)] = make_int2(ref[c], t);
            ref[c] = t;
        }
    float v[6][4];
    int r[4];
    for (int c = 0; c < 4; ++c) {
        const bool on = c < cnt;
        v[0][c] = on ? lo[c].x : FLT_MAX;
        v[1][c] = on ? hi[c].x : -FLT_MAX;
        v[2][c] = on ? lo[c].y : FLT_MAX;
        v[3][c] = on ? hi[c].y : -FLT_MAX;
        v[4][c] = on ? lo[c].z : FLT_MAX;
        v[5][c] = on ? hi[c].z : -FLT_MAX;
        r[c] = on ? ref[c] : kEmptyRef;
    }
    float4* o = nodes4 + (size_t)kNode4Float4 * job.y;
    for (int k = 0; k < 6; ++k) o[k] = make_float4(v[k][0], v[k][1], v[k][2], v[k][3]);
    o[6] = make_float4(__int_as_float(r[0]), __int_as_float(r[1]), __int_as_float(r[2]), __int_as_float(r[3]));
    o[7] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void __launch_bounds__(kThreads) k_collapse4(const float4* nodes2, const int2* qin, int nin, int2* qout,
                                                        int* nout, int* count4, float4* nodes4)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < nin) collapse4_one(nodes2, qin[w], qout, nout, count4, nodes4);
}

// ---------------------------------------------------------------- single-block build of small meshes
// A mesh of at most kSmallBuild triangles is too small to fill the GPU, and
// the per-round launches and host reads of the clustering would dominate its
// build. One block of kSmallThreads threads runs the same steps with barriers
// between them: the Morton sort (bitonic network on (key, index) pairs in
// shared memory, which gives the order of the stable radix sort), the PLOC
// rounds (same nearest-neighbour, merge and compaction functions) and the
// pointer-jumping positions; the 4-wide collapse runs its levels the same way.
constexpr int kSmallThreads = 1024;
constexpr int kSmallBuild = 16384;  // 12 bytes per triangle of shared memory for the sort

struct SmallBuild {
    const unsigned long long* keys;  // Morton keys of the triangles (unsorted)
    const unsigned* vals;            // their triangle ids
    const float4* tbox;
    int n, leaf_max, radius;
    float c_t, c_i;
    Clusters cl[2];
    int* nn;
    unsigned* keep;
    unsigned* pos;
    PlocNodes g;
    int* par[2];
    int* rel[2];
    int* noff;
    unsigned* perm;
    int* err;  // bit 4: the clustering did not converge
};

// exclusive scan of in[0..m) into out over the whole block; returns the total
__device__ unsigned block_exclusive_scan(const unsigned* in, unsigned* out, int m, unsigned* s_part)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, n_warps = blockDim.x >> 5;
    const int per = (m + blockDim.x - 1) / blockDim.x;
    const int b0 = min(m, tid * per), b1 = min(m, b0 + per);
    unsigned sum = 0;
    for (int k = b0; k < b1; ++k) sum += in[k];
    unsigned x = sum;  // inclusive scan over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_part[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < n_warps ? s_part[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_part[lane] = w;  // inclusive over the warps
    }
    __syncthreads();
    unsigned pre = x - sum + (warp > 0 ? s_part[warp - 1] : 0u);
    for (int k = b0; k < b1; ++k) {
        out[k] = pre;
        pre += in[k];
    }
    const unsigned total = s_part[n_warps - 1];
    __syncthreads();  // s_part is reused by the next call
    return total;
}

__global__ void __launch_bounds__(kSmallThreads) k_build_small(const SmallBuild b)
{
    extern __shared__ unsigned long long s_key[];  // [n] keys, then [n] triangle ids
    __shared__ unsigned s_part[32];
    __shared__ int s_m, s_next;
    const int tid = threadIdx.x, nt = blockDim.x, n = b.n;
    unsigned* s_val = reinterpret_cast<unsigned*>(s_key + n);
    for (int i = tid; i < n; i += nt) {
        s_key[i] = b.keys[i];
        s_val[i] = b.vals[i];
    }
    __syncthreads();
    // ascending by (key, id): bitonic merges over the next power of two; the
    // first step of each merge compares mirrored positions, so pairs reaching
    // past n (virtual +infinity) are already in order and are skipped
    int P = 1;
    while (P < n) P <<= 1;
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < (P >> 1); i += nt) {
                const int blk = i / j, off = i - blk * j;
                const int a = (j == (k >> 1)) ? blk * k + off : blk * 2 * j + off;
                const int c = (j == (k >> 1)) ? blk * k + k - 1 - off : a + j;
                if (c < n) {
                    const unsigned long long ka = s_key[a], kc = s_key[c];
                    const unsigned va = s_val[a], vc = s_val[c];
                    if (ka > kc || (ka == kc && va > vc)) {
                        s_key[a] = kc;
                        s_key[c] = ka;
                        s_val[a] = vc;
                        s_val[c] = va;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < n; i += nt) ploc_init_one(i, s_val, b.tbox, b.c_i, b.cl[0]);
    if (tid == 0) {
        s_m = n;
        s_next = n - 2;
    }
    __syncthreads();
    int cur = 0;
    for (int round = 0;; ++round) {
        const int m = s_m;  // the same in every thread: read after a barrier
        if (m <= 1) break;
        if (round >= (1 << 16)) {  // every round merges at least one pair
            if (tid == 0) atomicOr(b.err, 4);
            break;
        }
        for (int i = tid; i < m; i += nt) ploc_nn_one(i, m, b.radius, b.cl[cur], b.nn);
        __syncthreads();
        for (int i = tid; i < m; i += nt)
            ploc_merge_one(i, n, b.cl[cur], b.nn, &s_next, b.g, b.keep, b.leaf_max, b.c_t, b.c_i);
        __syncthreads();
        const unsigned total = block_exclusive_scan(b.keep, b.pos, m, s_part);
        for (int i = tid; i < m; i += nt) ploc_compact_one(i, b.cl[cur], b.keep, b.pos, b.cl[cur ^ 1]);
        __syncthreads();
        if (tid == 0) s_m = (int)total;
        cur ^= 1;
        __syncthreads();
    }
    int jr = 1;
    while ((1 << jr) < n) ++jr;
    int pj = 0;
    for (int r = 0; r <= jr; ++r, pj ^= 1) {
        for (int x = tid; x < 2 * n - 1; x += nt) ploc_jump_one(x, b.par[pj], b.rel[pj], b.par[pj ^ 1], b.rel[pj ^ 1]);
        __syncthreads();
    }
    for (int x = tid; x < 2 * n - 1; x += nt) ploc_positions_one(x, n, b.rel[pj], b.noff, b.perm);
}

// counters[0]: 4-wide nodes allocated; [1]: next-level queue length; [2]: 1 if too deep
__global__ void __launch_bounds__(kSmallThreads) k_collapse4_small(const float4* nodes2, int2* qa, int2* qb,
                                                                   int* counters, float4* nodes4)
{
    __shared__ int s_nin;
    if (threadIdx.x == 0) {
        qa[0] = make_int2(0, 0);
        counters[0] = 1;
        counters[1] = 0;
        counters[2] = 0;
        s_nin = 1;
    }
    __syncthreads();
    int2 *qi = qa, *qo = qb;
    for (int level = 0;; ++level) {
        const int nin = s_nin;
        if (nin <= 0) break;
        if (level > 4096) {  // deeper than any binary tree of < 2^27 leaves
            if (threadIdx.x == 0) counters[2] = 1;
            break;
        }
        for (int w = threadIdx.x; w < nin; w += blockDim.x) collapse4_one(nodes2, qi[w], qo, counters + 1, counters, nodes4);
        __syncthreads();
        if (threadIdx.x == 0) {
            s_nin = counters[1];
            counters[1] = 0;
        }
        __syncthreads();
        int2* t = qi;
        qi = qo;
        qo = t;
    }
}

// ---------------------------------------------------------------- octant copies
__global__ void __launch_bounds__(kThreads) k_octant_nodes(const float4* nodes, long long n_nodes, float4* out)
{
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n_nodes) return;
    const float4 n0 = nodes[4 * k], n1 = nodes[4 * k + 1], n2 = nodes[4 * k + 2], n3 = nodes[4 * k + 3];
    // (lo, hi) per axis: L x = n0.xy, L y = n0.zw, L z = n2.xy; R x = n1.xy, R y = n1.zw, R z = n2.zw
    const float Llo[3] = {n0.x, n0.z, n2.x}, Lhi[3] = {n0.y, n0.w, n2.y};
    const float Rlo[3] = {n1.x, n1.z, n2.z}, Rhi[3] = {n1.y, n1.w, n2.w};
    for (int o = 0; o < 8; ++o) {
        float Ln[3], Lf[3], Rn[3], Rf[3];
        for (int a = 0; a < 3; ++a) {
            const bool neg = (o >> a) & 1;
            Ln[a] = neg ? Lhi[a] : Llo[a];
            Lf[a] = neg ? Llo[a] : Lhi[a];
            Rn[a] = neg ? Rhi[a] : Rlo[a];
            Rf[a] = neg ? Rlo[a] : Rhi[a];
        }
        float4* d = out + 4 * ((long long)o * n_nodes + k);
        d[0] = make_float4(Ln[0], Ln[1], Ln[2], Rn[0]);
        d[1] = make_float4(Rn[1], Rn[2], Lf[0], Lf[1]);
        d[2] = make_float4(Lf[2], Rf[0], Rf[1], Rf[2]);
        d[3] = n3;
    }
}

struct Carve {
    char* p;
    size_t off, cap;
    template <class T>
    T* take(size_t count)
    {
        size_t o = (off + 255) & ~(size_t)255;
        off = o + count * sizeof(T);
        return (T*)(p + o);
    }
};

// ---------------------------------------------------------------- depth-first relayout
// The builders leave max(n - 1, 1) node slots, and the slots of clusters that
// the SAH collapse turned into leaves are never reached. The reachable nodes are
// renumbered in depth-first order, the child with the larger box first (the one
// a ray enters more often): a node's subtree becomes one contiguous range that
// starts right after it, and the tree shrinks to its reachable part. The root
// stays node 0; leaf references and boxes are unchanged, so every traversal
// visits the same boxes in the same order.

// parent of every internal child, as 2 * parent + side
__global__ void __launch_bounds__(kThreads) k_rl_parent(const float4* nodes, int m, int* parent)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const float4 r = nodes[4 * (size_t)i + 3];
    const int c0 = __float_as_int(r.x), c1 = __float_as_int(r.y);
    if (c0 >= 0 && c0 < m) parent[c0] = 2 * i;
    if (c1 >= 0 && c1 < m) parent[c1] = 2 * i + 1;
}

// internal nodes in each subtree, bottom-up from the nodes without internal
// children; the last child to arrive at a node finishes it
__global__ void __launch_bounds__(kThreads) k_rl_size(const float4* nodes, int m, const int* parent, int* arrive,
                                                      int* size)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const float4 r = nodes[4 * (size_t)i + 3];
    if (__float_as_int(r.x) >= 0 || __float_as_int(r.y) >= 0) return;
    size[i] = 1;
    __threadfence();
    int x = i;
    // a walk to the root passes at most m nodes; the bound guards against a malformed hierarchy
    for (int steps = 0; steps < m; ++steps) {
        const int pp = parent[x];
        if (pp < 0) return;
        const int p = pp >> 1;
        const float4 q = nodes[4 * (size_t)p + 3];
        const int l = __float_as_int(q.x), rr = __float_as_int(q.y);
        const int need = (l >= 0 ? 1 : 0) + (rr >= 0 ? 1 : 0);
        if (atomicAdd(arrive + p, 1) + 1 < need) return;  // the sibling finishes the node
        __threadfence();
        size[p] = 1 + (l >= 0 ? __ldcg(size + l) : 0) + (rr >= 0 ? __ldcg(size + rr) : 0);
        __threadfence();
        x = p;
    }
}

// side (0 left, 1 right) whose child comes first: the larger surface area
__device__ __forceinline__ int rl_first(const float4* nodes, int p)
{
    const float4 n0 = nodes[4 * (size_t)p], n1 = nodes[4 * (size_t)p + 1], n2 = nodes[4 * (size_t)p + 2];
    const float4 llo = make_float4(n0.x, n0.z, n2.x, 0.f), lhi = make_float4(n0.y, n0.w, n2.y, 0.f);
    const float4 rlo = make_float4(n1.x, n1.z, n2.z, 0.f), rhi = make_float4(n1.y, n1.w, n2.w, 0.f);
    return area(llo, lhi) >= area(rlo, rhi) ? 0 : 1;
}

// depth-first position of every reachable node (-1: not reachable from the root)
__global__ void __launch_bounds__(kThreads) k_rl_pos(const float4* nodes, int m, const int* parent, const int* size,
                                                     int* newpos)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int pos = 0, x = i, steps = 0;
    for (; steps < m; ++steps) {
        const int pp = parent[x];
        if (pp < 0) break;
        const int p = pp >> 1, side = pp & 1, f = rl_first(nodes, p);
        pos += 1;
        if (side != f) {
            const int c = __float_as_int(f == 0 ? nodes[4 * (size_t)p + 3].x : nodes[4 * (size_t)p + 3].y);
            if (c >= 0) pos += size[c];
        }
        x = p;
    }
    newpos[i] = (x == 0 && steps < m) ? pos : -1;
}

__global__ void __launch_bounds__(kThreads) k_rl_scatter(const float4* nodes, int m, const int* newpos, float4* out,
                                                         const int* size, int* n_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && n_out) *n_out = size[0];
    if (i >= m) return;
    const int q = newpos[i];
    if (q < 0) return;
    const float4 r = nodes[4 * (size_t)i + 3];
    int c0 = __float_as_int(r.x), c1 = __float_as_int(r.y);
    if (c0 >= 0) c0 = newpos[c0];
    if (c1 >= 0) c1 = newpos[c1];
    out[4 * (size_t)q] = nodes[4 * (size_t)i];
    out[4 * (size_t)q + 1] = nodes[4 * (size_t)i + 1];
    out[4 * (size_t)q + 2] = nodes[4 * (size_t)i + 2];
    out[4 * (size_t)q + 3] = make_float4(__int_as_float(c0), __int_as_float(c1), 0.f, 0.f);
}

}  // namespace

// Renumber the m node slots of b.nodes in depth-first order (the kernels
// above) through scratch taken from cv; *b.n_nodes_out gets the node count.
cudaError_t relayout(const BvhBuild& b, int m, Carve& cv, cudaStream_t st)
{
    int* parent = cv.take<int>(m);
    int* arrive = cv.take<int>(m);
    int* size = cv.take<int>(m);
    int* newpos = cv.take<int>(m);
    float4* tmp = cv.take<float4>(4 * (size_t)m);
    if (cv.off > cv.cap) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(parent, 0xFF, sizeof(int) * (size_t)m, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(arrive, 0, sizeof(int) * (size_t)m, st);
    if (e != cudaSuccess) return e;
    const int gm = (m + kThreads - 1) / kThreads;
    k_rl_parent<<<gm, kThreads, 0, st>>>(b.nodes, m, parent);
    k_rl_size<<<gm, kThreads, 0, st>>>(b.nodes, m, parent, arrive, size);
    k_rl_pos<<<gm, kThreads, 0, st>>>(b.nodes, m, parent, size, newpos);
    k_rl_scatter<<<gm, kThreads, 0, st>>>(b.nodes, m, newpos, tmp, size, b.n_nodes_out);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.nodes, tmp, sizeof(float4) * 4 * (size_t)m, cudaMemcpyDeviceToDevice, st);
    return e;
}

size_t bvh_scratch_bytes(long long n_tri)
{
    size_t n = (size_t)(n_tri < 2 ? 2 : n_tri);
    size_t nb = (n + kRsTile - 1) / kRsTile;
    size_t b = 0;
    auto add = [&](size_t bytes) { b = ((b + 255) & ~(size_t)255) + bytes; };
    add(64);                                // acc
    add(n * 32);                            // tbox
    add(n * 16);                            // cen
    add(n * 8); add(n * 8);                 // keys x2
    add(n * 4); add(n * 4);                 // vals x2
    add(256 * nb * 4);                      // hist
    add(scan_scratch_bytes(256 * (long long)nb));
    for (int k = 0; k < 6; ++k) add(n * 4); // left right first last par_int par_leaf
    add(n * 4);                             // flags
    add(n * 32); add(n * 32);               // lbox nbox
    add(n * 4); add(n * 4); add(n * 4);     // ncnt ncost ncol
    for (int k = 0; k < 2; ++k) {           // PLOC clusters, two buffers
        add(n * 16); add(n * 16); add(n * 4); add(n * 4); add(n * 4);
    }
    add(n * 4); add(n * 4); add(n * 4);     // nn keep pos
    add(scan_scratch_bytes((long long)n));
    add(n * 4); add(n * 4);                 // noff perm
    for (int k = 0; k < 4; ++k) add(2 * n * 4);  // parent links and offsets, two buffers each
    add(64);                                // counters
    for (int k = 0; k < 4; ++k) add(n * 4); // relayout: parent, arrivals, subtree sizes, new positions
    add(n * 64);                            // relayout: the renumbered nodes
    return b + 256;
}

cudaError_t bvh_build(const BvhBuild& b, cudaStream_t st)
{
    const int n = (int)b.n_tri;
    if (n < 1) return cudaErrorInvalidValue;
    Carve cv{(char*)b.scratch, 0, b.scratch_bytes};
    const int nn = n < 2 ? 2 : n;
    unsigned* acc = cv.take<unsigned>(16);
    float4* tbox = cv.take<float4>(2 * (size_t)nn);
    float4* cen = cv.take<float4>(nn);
    unsigned long long* k0 = cv.take<unsigned long long>(nn);
    unsigned long long* k1 = cv.take<unsigned long long>(nn);
    unsigned* v0 = cv.take<unsigned>(nn);
    unsigned* v1 = cv.take<unsigned>(nn);
    const int nb = (nn + kRsTile - 1) / kRsTile;
    unsigned* hist = cv.take<unsigned>(256 * (size_t)nb);
    void* sscr = cv.take<char>(scan_scratch_bytes(256 * (long long)nb));
    int* left = cv.take<int>(nn);
    int* right = cv.take<int>(nn);
    int* first = cv.take<int>(nn);
    int* last = cv.take<int>(nn);
    int* par_int = cv.take<int>(nn);
    int* par_leaf = cv.take<int>(nn);
    int* flags = cv.take<int>(nn);
    float4* lbox = cv.take<float4>(2 * (size_t)nn);
    float4* nbox = cv.take<float4>(2 * (size_t)nn);
    int* ncnt = cv.take<int>(nn);
    float* ncost = cv.take<float>(nn);
    int* ncol = cv.take<int>(nn);
    Clusters cl[2];
    for (int k = 0; k < 2; ++k) {
        cl[k].lo = cv.take<float4>(nn);
        cl[k].hi = cv.take<float4>(nn);
        cl[k].ref = cv.take<int>(nn);
        cl[k].cnt = cv.take<int>(nn);
        cl[k].cost = cv.take<float>(nn);
    }
    int* pnn = cv.take<int>(nn);
    unsigned* keep = cv.take<unsigned>(nn);
    unsigned* pos = cv.take<unsigned>(nn);
    void* pscan = cv.take<char>(scan_scratch_bytes((long long)nn));
    int* noff = cv.take<int>(nn);
    unsigned* perm = cv.take<unsigned>(nn);
    int* par[2];
    int* rel[2];
    for (int k = 0; k < 2; ++k) {
        par[k] = cv.take<int>(2 * (size_t)nn);
        rel[k] = cv.take<int>(2 * (size_t)nn);
    }
    int* ctr = cv.take<int>(16);
    if (cv.off > cv.cap) return cudaErrorInvalidValue;

    const int g = (n + kThreads - 1) / kThreads;
    k_acc_init<<<1, 32, 0, st>>>(acc, b.err_flag);
    int gv = (int)((b.n_vert + kThreads - 1) / kThreads);
    if (gv > 4096) gv = 4096;
    k_vertex_box<<<gv, kThreads, 0, st>>>(b.xyz, b.n_vert, acc, b.err_flag);
    k_prep<<<g, kThreads, 0, st>>>(b.xyz, b.tri, b.n_vert, n, tbox, cen, acc, b.err_flag);
    k_morton<<<g, kThreads, 0, st>>>(cen, n, acc, k0, v0, b.bbox_out);
    if (b.builder == 1 && n > 1 && n <= kSmallBuild) {
        const int nx = 2 * n - 1;
        cudaError_t e = cudaMemsetAsync(par[0], 0xFF, sizeof(int) * (size_t)nx, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(rel[0], 0, sizeof(int) * (size_t)nx, st);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_build_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(12 * (size_t)kSmallBuild));
        if (e != cudaSuccess) return e;
        SmallBuild sb;
        sb.keys = k0;
        sb.vals = v0;
        sb.tbox = tbox;
        sb.n = n;
        sb.leaf_max = b.leaf_max;
        sb.radius = b.radius > 0 ? b.radius : 16;
        sb.c_t = b.c_t;
        sb.c_i = b.c_i;
        sb.cl[0] = cl[0];
        sb.cl[1] = cl[1];
        sb.nn = pnn;
        sb.keep = keep;
        sb.pos = pos;
        sb.g = {left, right, nbox, ncnt, ncost, ncol, par[0], rel[0]};
        sb.par[0] = par[0];
        sb.par[1] = par[1];
        sb.rel[0] = rel[0];
        sb.rel[1] = rel[1];
        sb.noff = noff;
        sb.perm = perm;
        sb.err = b.err_flag;
        k_build_small<<<1, kSmallThreads, 12 * (size_t)n, st>>>(sb);
        k_ploc_emit<<<(n - 1 + kThreads - 1) / kThreads, kThreads, 0, st>>>(n, left, right, nbox, ncnt, ncol, noff,
                                                                            tbox, b.nodes);
        e = relayout(b, n - 1, cv, st);
        if (e != cudaSuccess) return e;
        k_reorder<<<g, kThreads, 0, st>>>(b.xyz, b.tri, b.n_vert, perm, n, b.tris, b.tri_nrm, b.tri_v12, b.tri_pos);
        return cudaGetLastError();
    }
    unsigned long long *ki = k0, *ko = k1;
    unsigned *vi = v0, *vo = v1;
    for (int pass = 0; pass < 8; ++pass) {
        k_rs_hist<<<nb, kRsThreads, 0, st>>>(ki, n, 8 * pass, hist, nb);
        cudaError_t e = scan_exclusive_u32(hist, hist, 256 * (long long)nb, false, nullptr, sscr, st);
        if (e != cudaSuccess) return e;
        k_rs_scatter<<<nb, kRsThreads, 0, st>>>(ki, vi, ko, vo, n, 8 * pass, hist, nb);
        unsigned long long* tk = ki; ki = ko; ko = tk;
        unsigned* tv = vi; vi = vo; vo = tv;
    }
    // after an even number of passes the sorted data is back in (k0, v0)
    if (b.builder == 1 && n > 1) {
        // PLOC over the Morton order; the live-cluster count stays on the device and the host reads it every
        // kRoundsPerSync rounds (extra rounds after the last merge change nothing)
        constexpr int kRoundsPerSync = 4;
        const float c_t = b.c_t, c_i = b.c_i;
        const int radius = b.radius > 0 ? b.radius : 16;
        const int nx = 2 * n - 1;
        k_ploc_init<<<g, kThreads, 0, st>>>(vi, tbox, n, c_i, cl[0]);
        int h[2] = {n - 2, n};  // next node id, live clusters
        cudaError_t e = cudaMemcpyAsync(ctr, h, sizeof(h), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(par[0], 0xFF, sizeof(int) * (size_t)nx, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(rel[0], 0, sizeof(int) * (size_t)nx, st);
        const PlocNodes pg = {left, right, nbox, ncnt, ncost, ncol, par[0], rel[0]};
        int m = n, cur = 0;
        for (int round = 0; e == cudaSuccess && m > 1; round += kRoundsPerSync) {
            if (round >= 1 << 16) return cudaErrorInvalidValue;  // every round merges at least one pair
            const int gm = (m + kThreads - 1) / kThreads;
            for (int r = 0; r < kRoundsPerSync && e == cudaSuccess; ++r) {
                k_ploc_nn<<<gm, kThreads, 0, st>>>(ctr + 1, radius, cl[cur], pnn);
                k_ploc_merge<<<gm, kThreads, 0, st>>>(ctr + 1, m, n, cl[cur], pnn, ctr, pg, keep, b.leaf_max, c_t, c_i);
                e = scan_exclusive_u32(keep, pos, m, false, (unsigned*)(ctr + 1), pscan, st);
                if (e != cudaSuccess) break;
                k_ploc_compact<<<gm, kThreads, 0, st>>>(m, cl[cur], keep, pos, cl[cur ^ 1]);
                e = cudaGetLastError();
                cur ^= 1;
            }
            if (e == cudaSuccess) e = cudaMemcpyAsync(&m, ctr + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
        if (e != cudaSuccess) return e;
        // first positions: pointer jumping over parent links (depth <= n - 1 < 2^rounds)
        int jr = 1;
        while ((1ll << jr) < (long long)n) ++jr;
        const int gx = (nx + kThreads - 1) / kThreads;
        int pj = 0;
        for (int r = 0; r <= jr; ++r, pj ^= 1)
            k_ploc_jump<<<gx, kThreads, 0, st>>>(nx, par[pj], rel[pj], par[pj ^ 1], rel[pj ^ 1]);
        k_ploc_positions<<<gx, kThreads, 0, st>>>(n, rel[pj], noff, perm);
        k_ploc_emit<<<(n - 1 + kThreads - 1) / kThreads, kThreads, 0, st>>>(n, left, right, nbox, ncnt, ncol, noff,
                                                                            tbox, b.nodes);
        e = relayout(b, n - 1, cv, st);
        if (e != cudaSuccess) return e;
        k_reorder<<<g, kThreads, 0, st>>>(b.xyz, b.tri, b.n_vert, perm, n, b.tris, b.tri_nrm, b.tri_v12, b.tri_pos);
        return cudaGetLastError();
    }
    if (n > 1) {
        k_karras<<<(n - 1 + kThreads - 1) / kThreads, kThreads, 0, st>>>(ki, n, left, right, first, last, par_int,
                                                                         par_leaf);
        cudaMemsetAsync(flags, 0, sizeof(int) * (size_t)n, st);
    }
    k_refit<<<g, kThreads, 0, st>>>(vi, tbox, n, left, right, par_int, par_leaf, flags, lbox, nbox, ncnt, ncost, ncol,
                                    b.leaf_max, b.c_t, b.c_i);
    int ge = n > 1 ? (n - 1 + kThreads - 1) / kThreads : 1;
    k_emit<<<ge, kThreads, 0, st>>>(n, left, right, first, lbox, nbox, ncnt, ncol, b.nodes);
    cudaError_t e = relayout(b, n > 1 ? n - 1 : 1, cv, st);
    if (e != cudaSuccess) return e;
    k_reorder<<<g, kThreads, 0, st>>>(b.xyz, b.tri, b.n_vert, vi, n, b.tris, b.tri_nrm, b.tri_v12, b.tri_pos);
    return cudaGetLastError();
}

cudaError_t build_octant_nodes(const float4* nodes, long long n_nodes, float4* out, cudaStream_t st)
{
    if (n_nodes <= 0) return cudaErrorInvalidValue;
    k_octant_nodes<<<(unsigned)((n_nodes + kThreads - 1) / kThreads), kThreads, 0, st>>>(nodes, n_nodes, out);
    return cudaGetLastError();
}

cudaError_t bvh4_collapse(const float4* nodes2, long long n_nodes2, float4* nodes4, int2* queue_a, int2* queue_b,
                          int* counters, int* n_nodes4, cudaStream_t st)
{
    if (n_nodes2 <= kSmallBuild) {
        k_collapse4_small<<<1, kSmallThreads, 0, st>>>(nodes2, queue_a, queue_b, counters, nodes4);
        int h[3] = {0, 0, 0};
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, counters, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && h[2]) e = cudaErrorInvalidValue;
        if (e == cudaSuccess) *n_nodes4 = h[0];
        return e;
    }
    // counters[0]: 4-wide nodes allocated; counters[1]: next-level queue length
    const int2 root = make_int2(0, 0);
    const int one = 1;
    cudaError_t e = cudaMemcpyAsync(queue_a, &root, sizeof(int2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(counters, &one, sizeof(int), cudaMemcpyHostToDevice, st);
    int nin = 1;
    int2 *qi = queue_a, *qo = queue_b;
    for (int level = 0; e == cudaSuccess && nin > 0; ++level) {
        if (level > 4096) return cudaErrorInvalidValue;  // deeper than any binary tree of < 2^27 leaves
        e = cudaMemsetAsync(counters + 1, 0, sizeof(int), st);
        if (e != cudaSuccess) break;
        k_collapse4<<<(nin + kThreads - 1) / kThreads, kThreads, 0, st>>>(nodes2, qi, nin, qo, counters + 1,
                                                                          counters, nodes4);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&nin, counters + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        int2* t = qi;
        qi = qo;
        qo = t;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(n_nodes4, counters, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

}  // namespace sbr
