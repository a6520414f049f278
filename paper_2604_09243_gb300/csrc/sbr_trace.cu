// sbr_trace.cu -- multi-bounce ray transport (Algorithm 2 of the paper) as a
// wavefront of persistent kernels:
//   pass 0        primary rays generated from their index on the aperture grid
//                 (Eq. L1-L3), closest hit, one 32-bit hit mask per 32 rays
//   scan          exclusive popcount prefix of the masks = dense record slots
//   pass b >= 1   the live rays of the previous pass, compacted into a queue,
//                 take their next closest-hit query (skipping the triangle just
//                 left); rays that miss or reach B_max write their record
// Each hit applies the specular reflection d - 2 (d.n) n, the PEC field update
// E' = 2 (n.E) n - E and the origin offset eps along the normal (Sec. 4), and
// stores the ray-tube coefficients the PO sum needs if this hit is the last one.
//
// Warps fetch 32 rays at a time from a global counter, so the grid stays full
// while rays finish at different depths; the traversal keeps a per-thread
// stack of node references, visits the nearer child first and tests the
// triangles of a leaf in FP32 Moller-Trumbore form.
#include <float.h>
#include <limits.h>

#include <algorithm>

#include "sbr_internal.h"

namespace sbr {

namespace {

constexpr int kTraceThreads = 256;
// conservative slab test: exit distance scaled by 1 + 2*gamma_3 (robust traversal)
constexpr float kBoxGrow = 1.0000008f;
constexpr unsigned kFull = 0xffffffffu;

// trace flag bits (mirror of SBR_TRACE_* in sbr.h)
constexpr int kFlagLiteral = 1;
constexpr int kFlagEscape = 2;

// The closest candidate of a query. During the traversal its exact distance is
// known to lie in [lo, t]; its stored distance t32 (key) is computed only when
// another candidate's interval overlaps, and at the end (key_closest), which
// sets t = t32.
struct Hit {
    float t;    // upper bound of the closest candidate's exact distance (box culling); t32 after key_closest
    float lo;   // lower bound of its exact distance
    float key;  // its t32 once computed, else -1
    int k;      // its position in the reordered triangles (-1: none)
    int orig;   // its original index
};

__device__ __forceinline__ float safe_rcp(float x)
{
    const float tiny = 1e-20f;
    return __frcp_rn(fabsf(x) > tiny ? x : copysignf(tiny, x));
}

// Two fused multiply-adds in one packed FP32 instruction: (a.x b.x + c.x,
// a.y b.y + c.y), each lane rounded once as fmaf rounds it.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pc, pr;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\tmov.b64 pc, {%6, %7};\n\t"
        "fma.rn.f32x2 pr, pa, pb, pc;\n\tmov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}

// ---------------------------------------------------------------- two-float helpers
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void tf_add(float& hi, float& lo, float x)
{
    float s, e;
    two_sum(hi, x, s, e);
    e = __fadd_rn(e, lo);
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}
__device__ __forceinline__ void tf_add_tf(float& hi, float& lo, float xh, float xl)
{
    float s, e;
    two_sum(hi, xh, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, xl));
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}
// a . b as an unevaluated two-float sum (exact products, compensated sum)
__device__ __forceinline__ void tf_dot(const float* a, float3 b, float& hi, float& lo)
{
    float p0 = __fmul_rn(a[0], b.x), e0 = __fmaf_rn(a[0], b.x, -p0);
    float p1 = __fmul_rn(a[1], b.y), e1 = __fmaf_rn(a[1], b.y, -p1);
    float p2 = __fmul_rn(a[2], b.z), e2 = __fmaf_rn(a[2], b.z, -p2);
    float s, e, s2, f;
    two_sum(p0, p1, s, e);
    two_sum(s, p2, s2, f);
    float lo_ = __fadd_rn(__fadd_rn(e, f), __fadd_rn(__fadd_rn(e0, e1), e2));
    hi = __fadd_rn(s2, lo_);
    lo = __fsub_rn(lo_, __fsub_rn(hi, s2));
}

// ---------------------------------------------------------------- FP32 cross and dot products
// cross(a, b) = (fma(a.y, b.z, -(a.z b.y)), ...) and dot(a, b) = fma(a.x, b.x, fma(a.y, b.y, a.z b.z)):
// each fma one rounding, every other operation one IEEE round-to-nearest operation
__device__ __forceinline__ float3 cross_s(float3 a, float3 b)
{
    return make_float3(__fmaf_rn(a.y, b.z, -__fmul_rn(a.z, b.y)), __fmaf_rn(a.z, b.x, -__fmul_rn(a.x, b.z)),
                       __fmaf_rn(a.x, b.y, -__fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float dot_s(float3 a, float3 b)
{
    return __fmaf_rn(a.x, b.x, __fmaf_rn(a.y, b.y, __fmul_rn(a.z, b.z)));
}

// ---------------------------------------------------------------- exact triangle test
// Which triangle a ray hits is decided exactly: the ray o + t d (its FP32
// values) against the closed triangle of the FP32 vertices, t > 0. With the
// exact E1 = v1 - v0, E2 = v2 - v0 and S = o - v0,
//   det = E1.(d x E2), U = S.(d x E2), V = d.(S x E1), T = E2.(S x E1),
// the ray hits when det != 0 and, taken with the sign of det, U >= 0, V >= 0,
// W = det - U - V >= 0 and T > 0 (Moller-Trumbore form, inclusive edges).
// They are evaluated in FP32 on the record's rounded edges; a forward error
// bound (gamma_n analysis of the rounded inputs, cross and dot products,
// folded into the per-triangle constants bUV, bD and the ray's largest
// |S| component) says when every sign is certain. Tests left open are taken
// again with the origin moved along the ray next to the triangle (U and V do
// not change, and their bounds shrink to the triangle's own size), and what is
// still open in FP64 from the exact vertices.
constexpr float kU = 0x1p-24f;  // FP32 unit roundoff

// 0: certain miss; 1: certain hit, tc ~ T / det with |tc - t| <= et;
// 2: the sign of U, V or W is open (det and T certain); 3: det or T open.
// U0, V0, T0, det: the FP32 values; bU, bV, bD, bT: bounds of their errors.
__device__ __forceinline__ int filter_core(float U0, float V0, float T0, float det, float bU, float bV, float bD,
                                           float bT, float& tc, float& et)
{
    const bool neg = det < 0.f;
    const float U = neg ? -U0 : U0, V = neg ? -V0 : V0, T = neg ? -T0 : T0;
    const float ad = fabsf(det);
    if (!(ad > bD)) return 3;  // det's sign open
    const float W = __fsub_rn(__fsub_rn(ad, U), V);
    const float bW = __fmaf_rn(0x1.1p-23f, __fadd_rn(__fadd_rn(ad, fabsf(U)), fabsf(V)), __fadd_rn(__fadd_rn(bU, bV), bD));
    if (U < -bU || V < -bV || W < -bW || T < -bT) return 0;
    if (!(T > bT)) return 3;
    if (!(U > bU && V > bV && W > bW)) return 2;
    tc = __fdividef(T, ad);
    et = __fmaf_rn(5.f * kU, tc, 1.01f * __fdividef(__fmaf_rn(tc, bD, bT), __fsub_rn(ad, bD)));
    return 1;
}

__device__ __forceinline__ float3 abs3(float3 a) { return make_float3(fabsf(a.x), fabsf(a.y), fabsf(a.z)); }
// |a| x |b| with absolute values: (|a.y||b.z| + |a.z||b.y|, ...), non-negative
__device__ __forceinline__ float3 cross_abs(float3 a, float3 b)
{
    a = abs3(a);
    b = abs3(b);
    return make_float3(__fmaf_rn(a.y, b.z, __fmul_rn(a.z, b.y)), __fmaf_rn(a.z, b.x, __fmul_rn(a.x, b.z)),
                       __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}

// Forward error bounds (Higham's gamma_n analysis: each rounded input, cross
// and dot product adds at most u of the absolute values it combines):
//   |U - U*| <= 8.1 u |S|.(|d| x |e2|),  |V - V*| <= 8.1 u |d|.(|S| x |e1|),
//   |det - det*| <= 8.1 u |e1|.(|d| x |e2|),  |T - T*| <= 9.1 u |e2|.(|S| x |e1|),
// with the 0.1 u covering the rounding of the bounds themselves. The record's
// bUV and bD bound them through norms (24 u L |S|_max, 14 u L^2, and
// 28 u L^2 |S|_max for T): three operations instead of some twenty, tried first.
__device__ __forceinline__ int tri_filter(float4 A, float4 B, float4 C, float3 o, float3 d, float& tc, float& et)
{
    const float3 e1 = make_float3(B.x, B.y, B.z), e2 = make_float3(C.x, C.y, C.z);
    const float3 p = cross_s(d, e2);
    const float det = dot_s(e1, p);
    const float3 s = make_float3(__fsub_rn(o.x, A.x), __fsub_rn(o.y, A.y), __fsub_rn(o.z, A.z));
    const float3 qv = cross_s(s, e1);
    const float U0 = dot_s(s, p), V0 = dot_s(d, qv), T0 = dot_s(e2, qv);
    const float smax = fmaxf(fmaxf(fabsf(s.x), fabsf(s.y)), fabsf(s.z));
    const float bUV = __fmul_rn(smax, B.w);
    if (!(B.w > 0.f)) return 0;
    return filter_core(U0, V0, T0, det, bUV, bUV, C.w, __fmul_rn(2.f * smax, C.w), tc, et);
}

// the per-component bounds of a test the norm bounds left open
__device__ __forceinline__ int tri_filter_tight(float4 A, float4 B, float4 C, float3 o, float3 d, float& tc, float& et)
{
    const float3 e1 = make_float3(B.x, B.y, B.z), e2 = make_float3(C.x, C.y, C.z);
    const float3 p = cross_s(d, e2);
    const float det = dot_s(e1, p);
    const float3 s = make_float3(__fsub_rn(o.x, A.x), __fsub_rn(o.y, A.y), __fsub_rn(o.z, A.z));
    const float3 qv = cross_s(s, e1);
    const float U0 = dot_s(s, p), V0 = dot_s(d, qv), T0 = dot_s(e2, qv);
    const float3 pa = cross_abs(d, e2), qa = cross_abs(s, e1);
    const float3 as = abs3(s), ad3 = abs3(d), a1 = abs3(e1), a2 = abs3(e2);
    return filter_core(U0, V0, T0, det, 0x1.03p-21f * dot_s(as, pa), 0x1.03p-21f * dot_s(ad3, qa),
                       0x1.03p-21f * dot_s(a1, pa), 0x1.23p-21f * dot_s(a2, qa), tc, et);
}

// o + lam d - v of one component as sc, with |sc - exact| <= 3 u sa, sa = |sc| + |z|
// (lam d and o + lam d as exact two-float sums; only the last two additions round)
__device__ __forceinline__ void shift1(float o, float d, float v, float lam, float& sc, float& sa)
{
    const float P = __fmul_rn(lam, d), Pe = __fmaf_rn(lam, d, -P);
    float X, Xe;
    two_sum(o, P, X, Xe);
    const float Y = __fsub_rn(X, v), Z = __fadd_rn(Xe, Pe);
    sc = __fadd_rn(Y, Z);
    sa = __fadd_rn(fabsf(sc), fabsf(Z));
}

// The decision left open by tri_filter (code 2 or 3): bit 0 of the result is
// set on a hit (then tc = T / det in FP32), bit 1 when FP64 decided.
__device__ __noinline__ int tri_refine(const float4* __restrict__ rec, const float4* __restrict__ v12, int k, float3 o,
                                        float3 d, int code, float& tc)
{
    const float4 A = __ldg(rec + 3 * (size_t)k), B = __ldg(rec + 3 * (size_t)k + 1), C = __ldg(rec + 3 * (size_t)k + 2);
    if (code >= 4) {  // from the norm bounds: try the per-component ones first
        float et;
        code = tri_filter_tight(A, B, C, o, d, tc, et);
        if (code < 2) return code;
    }
    const float3 e1 = make_float3(B.x, B.y, B.z), e2 = make_float3(C.x, C.y, C.z);
    const float3 p = cross_s(d, e2);
    const float det = dot_s(e1, p);
    const float3 s0 = make_float3(__fsub_rn(o.x, A.x), __fsub_rn(o.y, A.y), __fsub_rn(o.z, A.z));
    const float T0 = dot_s(e2, cross_s(s0, e1));
    tc = __fdiv_rn(T0, det);
    const float lam = __fdividef(T0, det);  // any finite value keeps U and V; near t it makes S small
    if (code == 2 && isfinite(lam)) {
        float3 sc, sa;
        shift1(o.x, d.x, A.x, lam, sc.x, sa.x);
        shift1(o.y, d.y, A.y, lam, sc.y, sa.y);
        shift1(o.z, d.z, A.z, lam, sc.z, sa.z);
        const float3 q1 = cross_s(sc, e1);
        const float U0 = dot_s(sc, p), V0 = dot_s(d, q1);
        // |d| x |e2| and sa x |e1|, then bounds of det (8 u), U and V (9.5 u each)
        const float3 ad3 = make_float3(fabsf(d.x), fabsf(d.y), fabsf(d.z));
        const float3 a1 = make_float3(fabsf(e1.x), fabsf(e1.y), fabsf(e1.z));
        const float3 a2 = make_float3(fabsf(e2.x), fabsf(e2.y), fabsf(e2.z));
        const float3 pa = make_float3(__fmaf_rn(ad3.y, a2.z, __fmul_rn(ad3.z, a2.y)),
                                      __fmaf_rn(ad3.z, a2.x, __fmul_rn(ad3.x, a2.z)),
                                      __fmaf_rn(ad3.x, a2.y, __fmul_rn(ad3.y, a2.x)));
        const float3 qa = make_float3(__fmaf_rn(sa.y, a1.z, __fmul_rn(sa.z, a1.y)),
                                      __fmaf_rn(sa.z, a1.x, __fmul_rn(sa.x, a1.z)),
                                      __fmaf_rn(sa.x, a1.y, __fmul_rn(sa.y, a1.x)));
        const float bD = 0x1.02p-21f * dot_s(a1, pa);
        const float bU = 0x1.3p-21f * dot_s(sa, pa);
        const float bV = 0x1.3p-21f * dot_s(ad3, qa);
        const float ad = fabsf(det);
        if (ad > bD) {
            const bool neg = det < 0.f;
            const float U = neg ? -U0 : U0, V = neg ? -V0 : V0;
            const float W = __fsub_rn(__fsub_rn(ad, U), V);
            const float bW = __fmaf_rn(0x1.1p-23f, __fadd_rn(__fadd_rn(ad, fabsf(U)), fabsf(V)), bD + bU + bV);
            if (U < -bU || V < -bV || W < -bW) return 0;
            if (U > bU && V > bV && W > bW) return 1;
        }
    }
    // FP64 from the exact vertices: differences of FP32 values are exact, the
    // products and sums round at 2^-53, far inside the 1e-6 edge band
    const float4 P1 = __ldg(v12 + 2 * (size_t)k), P2 = __ldg(v12 + 2 * (size_t)k + 1);
    const double x0 = A.x, y0 = A.y, z0 = A.z;
    const double E1x = (double)P1.x - x0, E1y = (double)P1.y - y0, E1z = (double)P1.z - z0;
    const double E2x = (double)P2.x - x0, E2y = (double)P2.y - y0, E2z = (double)P2.z - z0;
    const double Sx = (double)o.x - x0, Sy = (double)o.y - y0, Sz = (double)o.z - z0;
    const double Dx = d.x, Dy = d.y, Dz = d.z;
    const double Px = Dy * E2z - Dz * E2y, Py = Dz * E2x - Dx * E2z, Pz = Dx * E2y - Dy * E2x;
    double dt = E1x * Px + E1y * Py + E1z * Pz;
    if (dt == 0.0) return 2;
    const double Qx = Sy * E1z - Sz * E1y, Qy = Sz * E1x - Sx * E1z, Qz = Sx * E1y - Sy * E1x;
    double U = Sx * Px + Sy * Py + Sz * Pz, V = Dx * Qx + Dy * Qy + Dz * Qz, T = E2x * Qx + E2y * Qy + E2z * Qz;
    tc = (float)(T / dt);
    if (dt < 0.0) {
        dt = -dt;
        U = -U;
        V = -V;
        T = -T;
    }
    return (U >= 0.0 && V >= 0.0 && (dt - U) - V >= 0.0 && T > 0.0) ? 3 : 2;
}

// a . b as an unevaluated two-float sum hi + lo (exact products, compensated sum)
__device__ __forceinline__ void tf_dot3(float3 a, float3 b, float& hi, float& lo)
{
    const float v[3] = {a.x, a.y, a.z};
    tf_dot(v, b, hi, lo);
}

// Hit distance stored with a hit: t32 = fl32(((v0 - o) . n) / (d . n)), the
// distance along the ray to the plane of the FP32 unit normal n through v0,
// rounded once. d.n as a two-float sum (exact products, compensated sum) and
// its reciprocal are taken once per (direction, triangle) -- once per (aspect,
// triangle) for the parallel primary rays; per origin o, v0 - o exactly as a
// two-float vector (TwoSum), the numerator (v0 - o).n as a two-float sum (its
// error relative to |v0 - o|, so short hops keep their precision), a quotient
// within a few units of the last place, its remainder and one correction.
struct PlaneKey {
    float3 n;
    float dh, dl, rd;
};

__device__ __forceinline__ PlaneKey plane_key(const float4* __restrict__ nrm, int k, float3 d)
{
    PlaneKey K;
    const float4 N = __ldg(nrm + k);
    K.n = make_float3(N.x, N.y, N.z);
    tf_dot3(d, K.n, K.dh, K.dl);
    K.rd = __frcp_rn(K.dh);
    return K;
}

// t32 for origin o and triangle vertex v0 (tfb when d.n is exactly 0)
__device__ __forceinline__ float plane_key_t(const PlaneKey& K, float3 v0, float3 o, float tfb)
{
    if (K.dh == 0.f) return tfb;
    float3 a, b;
    two_sum(v0.x, -o.x, a.x, b.x);
    two_sum(v0.y, -o.y, a.y, b.y);
    two_sum(v0.z, -o.z, a.z, b.z);
    float nh, nl;
    tf_dot3(a, K.n, nh, nl);
    nl = __fmaf_rn(b.x, K.n.x, __fmaf_rn(b.y, K.n.y, __fmaf_rn(b.z, K.n.z, nl)));
    const float q = __fmul_rn(nh, K.rd);
    const float r = __fadd_rn(__fmaf_rn(-q, K.dh, nh), __fmaf_rn(-q, K.dl, nl));
    return __fmaf_rn(r, K.rd, q);
}

// The triangle data a query reads (records, normals, exact vertices, counters)
// are those of the kernel's TraceArgs, read from its parameter space where
// needed rather than held in registers through the traversal.
using TriRefs = TraceArgs;

__device__ __forceinline__ const TraceArgs& tri_refs(const TraceArgs& a) { return a; }

// counting runs: one test left open by the filter, decided in FP64 or not
__device__ __forceinline__ void count_open(unsigned long long* stats, int r)
{
    atomicAdd(stats + kStatOpen, 1ull);
    if (r & 2) atomicAdd(stats + kStatFp64, 1ull);
}

// t32 of reordered triangle k and its error bound: |t32 - exact t| <= u t32
// (rounding) + u L / |d.n| (plane of n32 against the triangle's own), u L <= bUV / 24
__device__ __noinline__ float key_of(const TriRefs& tr, int k, float3 o, float3 d, float tfb, float& slack)
{
    const float4 A = __ldg(tr.tris + 3 * (size_t)k), B = __ldg(tr.tris + 3 * (size_t)k + 1);
    const PlaneKey K = plane_key(tr.tri_nrm, k, d);
    const float t = plane_key_t(K, make_float3(A.x, A.y, A.z), o, tfb);
    slack = __fmaf_rn(2.f * kU, fabsf(t), __fdividef(0.08f * B.w, fabsf(K.dh)));
    return t;
}

// Two candidates whose distance intervals overlap: their stored distances are
// computed and compared (rare; kept out of the traversal loop's registers).
__device__ __noinline__ void resolve_overlap(const TriRefs& tr, int k, int orig, float tc, float3 o, float3 d, Hit& h)
{
    float sl;
    if (h.key < 0.f) {
        h.key = key_of(tr, h.k, o, d, h.t, sl);
        h.t = __fadd_rn(h.key, sl);
        h.lo = __fsub_rn(h.key, sl);
    }
    const float t = key_of(tr, k, o, d, tc, sl);
    if (t < h.key || (t == h.key && orig < h.orig)) {
        h.key = t;
        h.t = __fadd_rn(t, sl);
        h.lo = __fsub_rn(t, sl);
        h.k = k;
        h.orig = orig;
    }
}

// The closest hit is the smallest (t32, original triangle index). A certain
// hit whose distance interval lies beyond the closest candidate's is dropped,
// one whose interval lies before it replaces it, and only when the two overlap
// are their stored distances computed and compared.
__device__ __forceinline__ void consider_hit(const TriRefs& tr, int k, int orig, float tc, float et, float3 o,
                                             float3 d, Hit& h)
{
    const float lo = __fsub_rn(tc, et), hi = __fadd_rn(tc, et);
    if (lo > h.t) return;
    if (h.k < 0 || hi < h.lo) {
        h.t = hi;
        h.lo = lo;
        h.key = -1.f;
        h.k = k;
        h.orig = orig;
        return;
    }
    resolve_overlap(tr, k, orig, tc, o, d, h);
}

// after the traversal: the closest hit's t32 in h.t
__device__ __forceinline__ void key_closest(const TriRefs& tr, float3 o, float3 d, Hit& h)
{
    if (h.k < 0) return;
    if (h.key < 0.f) {
        float sl;
        h.key = key_of(tr, h.k, o, d, 0.5f * (h.t + h.lo), sl);
    }
    h.t = h.key;
}

// The triangles of leaf `ref`
template <bool kCount>
__device__ __forceinline__ void leaf_test(const TriRefs& tr, int ref, float3 o, float3 d, int skip, Hit& h,
                                          unsigned& ntri)
{
    const int first = leaf_first(ref), cnt = leaf_count(ref);
    for (int q = 0; q < cnt; ++q) {
        const int k = first + q;
        if (kCount) ++ntri;
        if (k == skip) continue;
        const float4* tp = tr.tris + 3 * (size_t)k;
        const float4 A = __ldg(tp), B = __ldg(tp + 1), C = __ldg(tp + 2);
        float tc = 0.f, et = FLT_MAX;
        const int f = tri_filter(A, B, C, o, d, tc, et);
        if (f == 0) continue;
        if (f >= 2) {
            const int r = tri_refine(tr.tris, tr.tri_v12, k, o, d, f + 2, tc);
            if (kCount) count_open(tr.stats, r);
            if (!(r & 1)) continue;
            et = FLT_MAX;
        }
        consider_hit(tr, k, __float_as_int(A.w), tc, et, o, d, h);
    }
}

template <bool kCount, int kStack>
__device__ __forceinline__ void closest_hit(const float4* __restrict__ nodes, const TriRefs& tris, float3 o,
                                            float3 d, int skip, int limit, Hit& h, unsigned& nvis, unsigned& ntri,
                                            bool& overflow)
{
    int stack[kStack];
    const float3 inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    const float3 oi = make_float3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
    // the slab distances of a box coordinate pair (lo, hi) of one axis: one packed fma
    const float2 ix = make_float2(inv.x, inv.x), iy = make_float2(inv.y, inv.y), iz = make_float2(inv.z, inv.z);
    const float2 mx = make_float2(-oi.x, -oi.x), my = make_float2(-oi.y, -oi.y), mz = make_float2(-oi.z, -oi.z);
    h.t = FLT_MAX;
    h.k = -1;
    h.orig = INT_MAX;
    h.lo = FLT_MAX;
    h.key = -1.f;
    int sp = 0;
    int ref = 0;
    // a query visits every node and leaf at most once; the bound guards against
    // a malformed hierarchy (reported like a stack overflow)
    for (int it = 0;; ++it) {
        if (it >= limit) {
            overflow = true;
            break;
        }
        if (ref >= 0) {
            const float4* nd = nodes + 4 * (size_t)ref;
            const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
            if (kCount) ++nvis;
            const float tmax = h.t;
            const float2 ax = fma2(make_float2(n0.x, n0.y), ix, mx), ay = fma2(make_float2(n0.z, n0.w), iy, my);
            const float2 az = fma2(make_float2(n2.x, n2.y), iz, mz), bx = fma2(make_float2(n1.x, n1.y), ix, mx);
            const float2 by = fma2(make_float2(n1.z, n1.w), iy, my), bz = fma2(make_float2(n2.z, n2.w), iz, mz);
            float an = fmaxf(fmaxf(fminf(ax.x, ax.y), fminf(ay.x, ay.y)), fmaxf(fminf(az.x, az.y), 0.f));
            float af = fminf(fminf(fmaxf(ax.x, ax.y), fmaxf(ay.x, ay.y)), fminf(fmaxf(az.x, az.y), tmax));
            float bn = fmaxf(fmaxf(fminf(bx.x, bx.y), fminf(by.x, by.y)), fmaxf(fminf(bz.x, bz.y), 0.f));
            float bf = fminf(fminf(fmaxf(bx.x, bx.y), fmaxf(by.x, by.y)), fminf(fmaxf(bz.x, bz.y), tmax));
            const int lref = __float_as_int(n3.x), rref = __float_as_int(n3.y);
            const bool hl = an <= af * kBoxGrow;
            const bool hr = (bn <= bf * kBoxGrow) && (rref != kEmptyRef);
            if (hl && hr) {
                const bool lnear = an <= bn;
                if (sp < kStack) stack[sp++] = lnear ? rref : lref;
                else overflow = true;
                ref = lnear ? lref : rref;
                continue;
            }
            if (hl) { ref = lref; continue; }
            if (hr) { ref = rref; continue; }
        } else {
            leaf_test<kCount>(tris, ref, o, d, skip, h, ntri);
        }
        if (sp == 0) break;
        ref = stack[--sp];
    }
}

// Binary traversal over the octant copies of the nodes: the ray's direction
// signs pick the copy whose near and far slabs are already chosen, so a child
// test is 6 FMA and 6 min/max instead of 6 FMA and 12 min/max. The FMA is
// monotone in the box coordinate, so every slab value, accepted box and visit
// order equals the min/max form of closest_hit.
template <bool kCount, int kStack>
__device__ __forceinline__ void closest_hit_oct(const float4* __restrict__ octant_nodes, long long n_nodes,
                                                const TriRefs& tris, float3 o, float3 d, int skip,
                                                int limit, Hit& h, unsigned& nvis, unsigned& ntri, bool& overflow)
{
    int stack[kStack];
    const float3 inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    const float3 oi = make_float3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
    const int oct = (inv.x < 0.f ? 1 : 0) | (inv.y < 0.f ? 2 : 0) | (inv.z < 0.f ? 4 : 0);
    const float4* nodes = octant_nodes + 4 * (size_t)oct * (size_t)n_nodes;
    h.t = FLT_MAX;
    h.k = -1;
    h.orig = INT_MAX;
    h.lo = FLT_MAX;
    h.key = -1.f;
    int sp = 0;
    int ref = 0;
    for (int it = 0;; ++it) {
        if (it >= limit) {
            overflow = true;
            break;
        }
        if (ref >= 0) {
            const float4* nd = nodes + 4 * (size_t)ref;
            const float4 f0 = __ldg(nd), f1 = __ldg(nd + 1), f2 = __ldg(nd + 2), f3 = __ldg(nd + 3);
            if (kCount) ++nvis;
            const float tmax = h.t;
            const float an = fmaxf(fmaxf(fmaf(f0.x, inv.x, -oi.x), fmaf(f0.y, inv.y, -oi.y)),
                                   fmaxf(fmaf(f0.z, inv.z, -oi.z), 0.f));
            const float af = fminf(fminf(fmaf(f1.z, inv.x, -oi.x), fmaf(f1.w, inv.y, -oi.y)),
                                   fminf(fmaf(f2.x, inv.z, -oi.z), tmax));
            const float bn = fmaxf(fmaxf(fmaf(f0.w, inv.x, -oi.x), fmaf(f1.x, inv.y, -oi.y)),
                                   fmaxf(fmaf(f1.y, inv.z, -oi.z), 0.f));
            const float bf = fminf(fminf(fmaf(f2.y, inv.x, -oi.x), fmaf(f2.z, inv.y, -oi.y)),
                                   fminf(fmaf(f2.w, inv.z, -oi.z), tmax));
            const int lref = __float_as_int(f3.x), rref = __float_as_int(f3.y);
            const bool hl = an <= af * kBoxGrow;
            const bool hr = bn <= bf * kBoxGrow;
            if (hl && hr) {
                const bool lnear = an <= bn;
                if (sp < kStack) stack[sp++] = lnear ? rref : lref;
                else overflow = true;
                ref = lnear ? lref : rref;
                continue;
            }
            if (hl) { ref = lref; continue; }
            if (hr) { ref = rref; continue; }
        } else {
            leaf_test<kCount>(tris, ref, o, d, skip, h, ntri);
        }
        if (sp == 0) break;
        ref = stack[--sp];
    }
}

// 4-wide variant: the near and far slab of each axis are chosen once per ray
// from the sign of its direction, which gives the same FP32 values as the
// per-axis min / max of the binary test (the fused product is monotone in the
// box coordinate), so both trees accept exactly the same child boxes. Hit
// children are ordered near to far by a 5-exchange sorting network; the far
// ones go on the stack with their entry distance and are skipped when popped
// behind the closest hit so far.
__device__ __forceinline__ void cswap(float& ka, int& ra, float& kb, int& rb)
{
    const bool sw = kb < ka;
    const float k = sw ? kb : ka, k2 = sw ? ka : kb;
    const int r = sw ? rb : ra, r2 = sw ? ra : rb;
    ka = k;
    kb = k2;
    ra = r;
    rb = r2;
}

template <bool kCount, int kStack>
__device__ __forceinline__ void closest_hit4(const float4* __restrict__ nodes, const TriRefs& tris,
                                             float3 o, float3 d, int skip, int limit, Hit& h, unsigned& nvis,
                                             unsigned& ntri, bool& overflow)
{
    int stack[kStack];
    float stack_t[kStack];
    const float3 inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    const float3 oi = make_float3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
    // float4 index of the near slab of each axis inside a node (lo: even, hi: odd)
    const int sx = inv.x >= 0.f ? 0 : 1, sy = inv.y >= 0.f ? 2 : 3, sz = inv.z >= 0.f ? 4 : 5;
    h.t = FLT_MAX;
    h.k = -1;
    h.orig = INT_MAX;
    h.lo = FLT_MAX;
    h.key = -1.f;
    int sp = 0;
    int ref = 0;
    for (int it = 0;; ++it) {
        if (it >= limit) {
            overflow = true;
            break;
        }
        if (ref >= 0) {
            const float4* nd = nodes + (size_t)kNode4Float4 * ref;
            const float4 nx = __ldg(nd + sx), fx = __ldg(nd + (sx ^ 1)), ny = __ldg(nd + sy), fy = __ldg(nd + (sy ^ 1));
            const float4 nz = __ldg(nd + sz), fz = __ldg(nd + (sz ^ 1));
            const float4 rr = __ldg(nd + 6);
            if (kCount) ++nvis;
            const float tmax = h.t;
#define SBR_SLAB(c, tn, tf)                                                                                  \
    const float tn = fmaxf(fmaxf(fmaf(nx.c, inv.x, -oi.x), fmaf(ny.c, inv.y, -oi.y)),                       \
                           fmaxf(fmaf(nz.c, inv.z, -oi.z), 0.f));                                           \
    const float tf = fminf(fminf(fmaf(fx.c, inv.x, -oi.x), fmaf(fy.c, inv.y, -oi.y)),                       \
                           fminf(fmaf(fz.c, inv.z, -oi.z), tmax));
            SBR_SLAB(x, tn0, tf0)
            SBR_SLAB(y, tn1, tf1)
            SBR_SLAB(z, tn2, tf2)
            SBR_SLAB(w, tn3, tf3)
#undef SBR_SLAB
            int r0 = __float_as_int(rr.x), r1 = __float_as_int(rr.y), r2 = __float_as_int(rr.z),
                r3 = __float_as_int(rr.w);
            float k0 = (tn0 <= tf0 * kBoxGrow && r0 != kEmptyRef) ? tn0 : FLT_MAX;
            float k1 = (tn1 <= tf1 * kBoxGrow && r1 != kEmptyRef) ? tn1 : FLT_MAX;
            float k2 = (tn2 <= tf2 * kBoxGrow && r2 != kEmptyRef) ? tn2 : FLT_MAX;
            float k3 = (tn3 <= tf3 * kBoxGrow && r3 != kEmptyRef) ? tn3 : FLT_MAX;
            cswap(k0, r0, k1, r1);
            cswap(k2, r2, k3, r3);
            cswap(k0, r0, k2, r2);
            cswap(k1, r1, k3, r3);
            cswap(k1, r1, k2, r2);
            if (k0 == FLT_MAX) {
                ref = kEmptyRef;  // no child hit: pop
            } else {
                // push hits far to near (the nearest is visited now)
                if (k3 != FLT_MAX) {
                    if (sp < kStack) {
                        stack[sp] = r3;
                        stack_t[sp++] = k3;
                    } else {
                        overflow = true;
                    }
                }
                if (k2 != FLT_MAX) {
                    if (sp < kStack) {
                        stack[sp] = r2;
                        stack_t[sp++] = k2;
                    } else {
                        overflow = true;
                    }
                }
                if (k1 != FLT_MAX) {
                    if (sp < kStack) {
                        stack[sp] = r1;
                        stack_t[sp++] = k1;
                    } else {
                        overflow = true;
                    }
                }
                ref = r0;
                continue;
            }
        } else {
            leaf_test<kCount>(tris, ref, o, d, skip, h, ntri);
        }
        // pop, skipping entries that start behind the closest hit so far
        ref = kEmptyRef;
        while (sp > 0) {
            --sp;
            if (stack_t[sp] <= h.t * kBoxGrow) {
                ref = stack[sp];
                break;
            }
        }
        if (ref == kEmptyRef) break;
    }
}

// Warp-cooperative (packet) traversal of the binary tree: the 32 lanes walk
// one path together, so every node and leaf fetch is a single broadcast and
// the loop never diverges. Each lane carries a "wants" flag per node (and one
// bit per stack entry): it wants a node when its own ray enters the node's box,
// and it tests boxes and leaf triangles only for nodes it wants, so its
// result and its visit counts are those of its own ray. The warp descends into
// a child when any lane wants it; when both children are wanted, the one that
// most lanes reach first goes first. Must be called by all 32 lanes together.
template <bool kCount, int kStack>
__device__ __forceinline__ void closest_hit_packet(const float4* __restrict__ nodes, const TriRefs& tris,
                                                   bool active, float3 o, float3 d, int skip, int limit, Hit& h,
                                                   unsigned& nvis, unsigned& ntri, bool& overflow)
{
    static_assert(kStack <= 64, "packet stack flags are one 64-bit word");
    int stack[kStack];
    unsigned long long wb = 0;  // lane wants stack entry k: bit k
    const float3 inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    const float3 oi = make_float3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
    h.t = FLT_MAX;
    h.k = -1;
    h.orig = INT_MAX;
    h.lo = FLT_MAX;
    h.key = -1.f;
    int sp = 0;
    int ref = 0;
    bool want = active;
    bool ovf = false;
    for (int it = 0;; ++it) {
        if (it >= limit) {
            ovf = true;
            break;
        }
        if (ref >= 0) {
            const float4* nd = nodes + 4 * (size_t)ref;
            const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
            if (kCount && want) ++nvis;
            const float tmax = h.t;
            float ax0 = fmaf(n0.x, inv.x, -oi.x), ax1 = fmaf(n0.y, inv.x, -oi.x);
            float ay0 = fmaf(n0.z, inv.y, -oi.y), ay1 = fmaf(n0.w, inv.y, -oi.y);
            float az0 = fmaf(n2.x, inv.z, -oi.z), az1 = fmaf(n2.y, inv.z, -oi.z);
            float bx0 = fmaf(n1.x, inv.x, -oi.x), bx1 = fmaf(n1.y, inv.x, -oi.x);
            float by0 = fmaf(n1.z, inv.y, -oi.y), by1 = fmaf(n1.w, inv.y, -oi.y);
            float bz0 = fmaf(n2.z, inv.z, -oi.z), bz1 = fmaf(n2.w, inv.z, -oi.z);
            float an = fmaxf(fmaxf(fminf(ax0, ax1), fminf(ay0, ay1)), fmaxf(fminf(az0, az1), 0.f));
            float af = fminf(fminf(fmaxf(ax0, ax1), fmaxf(ay0, ay1)), fminf(fmaxf(az0, az1), tmax));
            float bn = fmaxf(fmaxf(fminf(bx0, bx1), fminf(by0, by1)), fmaxf(fminf(bz0, bz1), 0.f));
            float bf = fminf(fminf(fmaxf(bx0, bx1), fmaxf(by0, by1)), fminf(fmaxf(bz0, bz1), tmax));
            const int lref = __float_as_int(n3.x), rref = __float_as_int(n3.y);
            const bool hl = want && an <= af * kBoxGrow;
            const bool hr = want && (bn <= bf * kBoxGrow) && (rref != kEmptyRef);
            const unsigned ml = __ballot_sync(kFull, hl), mr = __ballot_sync(kFull, hr);
            if (ml && mr) {
                const unsigned both = ml & mr, lfirst = __ballot_sync(kFull, hl && hr && an <= bn);
                const bool goleft = both ? 2 * __popc(lfirst) >= __popc(both) : __popc(ml) >= __popc(mr);
                const int fref = goleft ? rref : lref;
                const bool wfar = goleft ? hr : hl;
                if (sp < kStack) {
                    stack[sp] = fref;
                    wb = wfar ? (wb | (1ull << sp)) : (wb & ~(1ull << sp));
                    ++sp;
                } else {
                    ovf = true;
                }
                ref = goleft ? lref : rref;
                want = goleft ? hl : hr;
                continue;
            }
            if (ml) {
                ref = lref;
                want = hl;
                continue;
            }
            if (mr) {
                ref = rref;
                want = hr;
                continue;
            }
        } else if (want) {
            leaf_test<kCount>(tris, ref, o, d, skip, h, ntri);
        }
        if (sp == 0) break;
        --sp;
        ref = stack[sp];
        want = (wb >> sp) & 1ull;
    }
    if (active && ovf) overflow = true;
}

// ---------------------------------------------------------------- per-ray state in registers
struct Ray {
    float3 o, d, ev;
    float lacc_hi, lacc_lo, cos0;
    float c[5];
    float lc_hi, lc_lo, nfs;
    int angle, local, last, nb;
};

// The live-ray queues, the records and the raster keys are each written once
// and read once: their loads and stores are marked evict-first (__ldcs /
// __stcs) so that they do not push the tree and the triangles out of L1 and L2.
__device__ __forceinline__ void load_state(const RayState* __restrict__ q, unsigned i, Ray& r)
{
    const float4* p = reinterpret_cast<const float4*>(q + i);
    float4 a = __ldcs(p), b = __ldcs(p + 1), c = __ldcs(p + 2), e = __ldcs(p + 3), f = __ldcs(p + 4);
    int4 g = __ldcs(reinterpret_cast<const int4*>(p) + 5);
    r.o = make_float3(a.x, a.y, a.z);
    r.d = make_float3(a.w, b.x, b.y);
    r.ev = make_float3(b.z, b.w, c.x);
    r.lacc_hi = c.y;
    r.lacc_lo = c.z;
    r.cos0 = c.w;
    r.c[0] = e.x; r.c[1] = e.y; r.c[2] = e.z; r.c[3] = e.w;
    r.c[4] = f.x;
    r.lc_hi = f.y;
    r.lc_lo = f.z;
    r.nfs = f.w;
    r.angle = g.x; r.local = g.y; r.last = g.z; r.nb = g.w;
}

// The traversal needs only the origin, the direction and the triangle to
// skip: load those first and the rest of the state after the query, so the
// payload does not occupy registers during the traversal.
__device__ __forceinline__ void load_geom(const RayState* __restrict__ q, unsigned i, Ray& r)
{
    const float4* p = reinterpret_cast<const float4*>(q + i);
    const float4 a = __ldcs(p), b = __ldcs(p + 1);
    r.o = make_float3(a.x, a.y, a.z);
    r.d = make_float3(a.w, b.x, b.y);
    r.last = __ldcs(reinterpret_cast<const int4*>(p) + 5).z;
}

__device__ __forceinline__ void load_payload(const RayState* __restrict__ q, unsigned i, Ray& r)
{
    const float4* p = reinterpret_cast<const float4*>(q + i);
    const float4 b = __ldcs(p + 1), c = __ldcs(p + 2), e = __ldcs(p + 3), f = __ldcs(p + 4);
    const int4 g = __ldcs(reinterpret_cast<const int4*>(p) + 5);
    r.ev = make_float3(b.z, b.w, c.x);
    r.lacc_hi = c.y;
    r.lacc_lo = c.z;
    r.cos0 = c.w;
    r.c[0] = e.x; r.c[1] = e.y; r.c[2] = e.z; r.c[3] = e.w;
    r.c[4] = f.x;
    r.lc_hi = f.y;
    r.lc_lo = f.z;
    r.nfs = f.w;
    r.angle = g.x; r.local = g.y; r.nb = g.w;
}

__device__ __forceinline__ void store_state(RayState* __restrict__ q, unsigned i, const Ray& r)
{
    float4* p = reinterpret_cast<float4*>(q + i);
    __stcs(p + 0, make_float4(r.o.x, r.o.y, r.o.z, r.d.x));
    __stcs(p + 1, make_float4(r.d.y, r.d.z, r.ev.x, r.ev.y));
    __stcs(p + 2, make_float4(r.ev.z, r.lacc_hi, r.lacc_lo, r.cos0));
    __stcs(p + 3, make_float4(r.c[0], r.c[1], r.c[2], r.c[3]));
    __stcs(p + 4, make_float4(r.c[4], r.lc_hi, r.lc_lo, r.nfs));
    __stcs(reinterpret_cast<int4*>(p) + 5, make_int4(r.angle, r.local, r.last, r.nb));
}

__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Update the ray at its closest hit: path, bounce count, candidate PO
// coefficients of this hit (used if it turns out to be the last), reflection,
// PEC field update and the new origin. The stored state is FP32, each value
// the rounding of its formula: x = fl32(o + t32 d), dn = fl32(d . n32),
// d' = fl32(d - 2 dn n32), o' = fl32(x + eps nf) (one fma each; dn from a
// compensated dot product).
__device__ __forceinline__ void apply_hit(const AngleDev& A, const float4* __restrict__ nrm, const Hit& h, int flags,
                                          Ray& r)
{
    const float3 x = make_float3(__fmaf_rn(h.t, r.d.x, r.o.x), __fmaf_rn(h.t, r.d.y, r.o.y),
                                 __fmaf_rn(h.t, r.d.z, r.o.z));
    tf_add(r.lacc_hi, r.lacc_lo, h.t);
    const int nb_before = r.nb;
    r.nb = nb_before + 1;
    const float4 N4 = __ldg(nrm + h.k);
    const float3 n = make_float3(N4.x, N4.y, N4.z);
    float dn, dnl;
    tf_dot3(r.d, n, dn, dnl);
    const float3 nf = dn < 0.f ? n : make_float3(-n.x, -n.y, -n.z);
    r.nfs = dn < 0.f ? 1.f : -1.f;
    const float adn = fabsf(dn);
    const float3 rh = make_float3(A.rhat[0], A.rhat[1], A.rhat[2]);
    if (r.nb == 1) r.cos0 = dot3(nf, rh);
    // candidate path L = k.o0 + sum t - r_rx.x (monostatic: r_rx = -k)
    float kh, kl;
    tf_dot(A.rxdir, x, kh, kl);
    r.lc_hi = r.lacc_hi;
    r.lc_lo = r.lacc_lo;
    tf_add_tf(r.lc_hi, r.lc_lo, kh, kl);
    // H-transmit field from the V one: E_H = s (d x E_V), s = +1 after an odd number of reflections
    const float sH = (nb_before & 1) ? 1.f : -1.f;
    const float3 eh = make_float3(sH * (r.d.y * r.ev.z - r.d.z * r.ev.y), sH * (r.d.z * r.ev.x - r.d.x * r.ev.z),
                                  sH * (r.d.x * r.ev.y - r.d.y * r.ev.x));
    const float dS = adn > 0.f ? __fdiv_rn(A.dA, adn) : 0.f;
    const float nfd = dot3(nf, r.d);
    // radiation toward the receiver, projected on its basis
    const float3 rr = make_float3(A.rxr[0], A.rxr[1], A.rxr[2]);
    const float3 vh = make_float3(A.rxv[0], A.rxv[1], A.rxv[2]);
    const float3 hh = make_float3(A.rxh[0], A.rxh[1], A.rxh[2]);
    float3 W[2];
    const float3 Eq[2] = {eh, r.ev};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const float ne = dot3(nf, Eq[q]);
        // J = 2 nf x (d x E) = 2 (d (nf.E) - E (nf.d))
        const float3 J = make_float3(2.f * (r.d.x * ne - Eq[q].x * nfd), 2.f * (r.d.y * ne - Eq[q].y * nfd),
                                     2.f * (r.d.z * ne - Eq[q].z * nfd));
        const float jr = dot3(J, rr);
        W[q] = make_float3(dS * (J.x - jr * rr.x), dS * (J.y - jr * rr.y), dS * (J.z - jr * rr.z));
    }
    r.c[0] = dot3(W[0], hh);  // HH
    r.c[1] = dot3(W[1], vh);  // VV
    r.c[2] = dot3(W[1], hh);  // HV
    r.c[3] = dot3(W[0], vh);  // VH
    const float gam = (r.nb & 1) ? -1.f : 1.f;  // Gamma^N, Gamma = -1
    r.c[4] = -2.f * A.dA * r.cos0 * gam;
    if (flags & kFlagLiteral) {
        // scalar form with e^{-j 2 k R}: L = 2 (k.o0 + R), stored in the candidate path
        r.lc_hi = 2.f * r.lacc_hi;
        r.lc_lo = 2.f * r.lacc_lo;
    }
    // PEC field update (FP32), then the stored reflection and offset origin
    const float nev = dot3(n, r.ev);
    r.ev = make_float3(fmaf(2.f * nev, n.x, -r.ev.x), fmaf(2.f * nev, n.y, -r.ev.y), fmaf(2.f * nev, n.z, -r.ev.z));
    const float m2 = -2.f * dn;
    r.d = make_float3(__fmaf_rn(m2, n.x, r.d.x), __fmaf_rn(m2, n.y, r.d.y), __fmaf_rn(m2, n.z, r.d.z));
    r.o = make_float3(__fmaf_rn(A.eps, nf.x, x.x), __fmaf_rn(A.eps, nf.y, x.y), __fmaf_rn(A.eps, nf.z, x.z));
    r.last = h.k;
}

__device__ __forceinline__ long long ray_global(const TraceArgs& a, const Ray& r)
{
    return a.ray_off[r.angle] + r.local;
}

// Rays are processed in tiles of W x H = 32 grid points (W = 2^tw_log2, 8 x 4
// by default): processing index p of an aspect maps to grid point
// (i, j) = (W bu + p % W, H bv + (p % 32) / W), tile p / 32 = bv * nbu + bu,
// so the 32 lanes of a warp trace a compact patch of the aperture.
__device__ __forceinline__ void tile_ij(const AngleDev& A, int p, int& i, int& j)
{
    const int blk = p >> 5, l = p & 31, tw = A.tw_log2;
    const int bv = blk / A.nbu, bu = blk - bv * A.nbu;
    i = (bu << tw) + (l & ((1 << tw) - 1));
    j = bv * (32 >> tw) + (l >> tw);
}

// Bistatic: the last hit contributes only if the receiver lies on the side of
// its oriented FP32 normal (the sign of the exact dot product) and a query from
// the offset origin toward the receiver meets no triangle (the one just hit is
// skipped).
__device__ __forceinline__ bool rx_visible(const TraceArgs& a, const AngleDev& A, const Ray& r, unsigned& nq,
                                           bool& ovf)
{
    const float4 N4 = __ldg(a.tri_nrm + r.last);
    const float3 n = make_float3(N4.x * r.nfs, N4.y * r.nfs, N4.z * r.nfs);
    const float3 rx = make_float3(A.rxr[0], A.rxr[1], A.rxr[2]);
    float sh, sl;
    tf_dot3(n, rx, sh, sl);  // the sign of the exact dot product
    if (!(sh > 0.f)) return false;
    Hit h;
    unsigned nv = 0, nt = 0;
    if (a.wide) closest_hit4<false, 64>(a.nodes, tri_refs(a), r.o, rx, r.last, a.visit_limit, h, nv, nt, ovf);
    else if (a.octant)
        closest_hit_oct<false, 64>(a.nodes, a.n_nodes, tri_refs(a), r.o, rx, r.last, a.visit_limit, h, nv, nt, ovf);
    else closest_hit<false, 64>(a.nodes, tri_refs(a), r.o, rx, r.last, a.visit_limit, h, nv, nt, ovf);
    ++nq;
    return h.k < 0;
}

__device__ __forceinline__ void emit(const TraceArgs& a, const Ray& r, bool zero)
{
    const long long g = ray_global(a, r);
    int i, j;
    const AngleDev& A = a.angles[r.angle];
    tile_ij(A, r.local, i, j);
    const int ray_id = j * A.nu + i;
    const long long tile = g >> 5;
    const unsigned bit = (unsigned)(g & 31);
    const unsigned slot = a.tile_base[tile] + __popc(a.mask[tile] & ((1u << bit) - 1u));
    Record* rec = a.rec_of ? a.rec + a.rec_of[r.angle] : a.rec;
    float4* p = reinterpret_cast<float4*>(rec + slot);
    if (zero) {
        __stcs(p + 0, make_float4(0.f, 0.f, 0.f, 0.f));
        __stcs(p + 1, make_float4(0.f, 0.f, 0.f, __int_as_float(ray_id)));
    } else {
        __stcs(p + 0, make_float4(r.c[0], r.c[1], r.c[2], r.c[3]));
        __stcs(p + 1, make_float4(r.c[4], r.lc_hi, r.lc_lo, __int_as_float(ray_id)));
    }
    if (a.hit_nb) a.hit_nb[g] = r.nb;
}

__device__ __forceinline__ void record_hit(const TraceArgs& a, const Ray& r, const Hit& h)
{
    if (!a.hit_tri) return;
    const long long g = ray_global(a, r);
    a.hit_tri[g * a.max_bounces + (r.nb - 1)] = h.orig;
    a.hit_t[g * a.max_bounces + (r.nb - 1)] = h.t;
}

__device__ __forceinline__ int find_angle(const long long* __restrict__ off, int n, long long g)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// warp-aggregated append of the lanes of m to queue q; every lane of the warp must call it
__device__ __forceinline__ void append(RayState* q, unsigned* count, unsigned m, const Ray& r)
{
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if ((m >> lane) & 1u) store_state(q, base + __popc(m & ((1u << lane) - 1u)), r);
}

// the rays that go on: to the live-ray queue, or to the ray pool while it has room
__device__ __forceinline__ void push(const TraceArgs& a, bool want, Ray& r)
{
    const unsigned m = __ballot_sync(kFull, want);
    if (!m) return;
    if (!a.pool) {
        append(a.q_out, a.q_out_count, m, r);
        return;
    }
    r.angle += a.angle_shift;  // the pool indexes the trace's aspects
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(a.pool_count, (unsigned)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    const unsigned idx = base + __popc(m & ((1u << lane) - 1u));
    const bool fit = want && idx < a.pool_cap;
    if (fit) store_state(a.pool, idx, r);
    const unsigned over = __ballot_sync(kFull, want && !fit);
    if (over) append(a.q_out, a.q_out_count, over, r);  // kept until the pool has been traced
}

template <bool kCount>
__device__ __forceinline__ void flush_stats(const TraceArgs& a, unsigned q, unsigned nvis, unsigned ntri, bool ovf,
                                            unsigned nhit = 0, unsigned nlist = 0, unsigned long long wvis = 0)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        q += __shfl_xor_sync(kFull, q, o);
        if (kCount) {
            nvis += __shfl_xor_sync(kFull, nvis, o);
            ntri += __shfl_xor_sync(kFull, ntri, o);
            nhit += __shfl_xor_sync(kFull, nhit, o);
            nlist += __shfl_xor_sync(kFull, nlist, o);
        }
    }
    const unsigned ov = __ballot_sync(kFull, ovf);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(a.stats + kStatQueries, (unsigned long long)q);
        if (kCount) {
            atomicAdd(a.stats + kStatNodes, (unsigned long long)nvis);
            atomicAdd(a.stats + kStatTris, (unsigned long long)ntri);
            if (nhit) atomicAdd(a.stats + kStatHits, (unsigned long long)nhit);
            if (nlist) atomicAdd(a.stats + kStatListed, (unsigned long long)nlist);
            if (wvis) atomicAdd(a.stats + kStatWarpNodes, wvis);
        }
        if (ov) atomicAdd(a.stats + kStatOverflow, (unsigned long long)__popc(ov));
    }
}

// One closest-hit query per lane. kMode 0: per-lane binary traversal; 1: per-lane
// 4-wide traversal; 2: warp-cooperative binary traversal (all 32 lanes call it);
// 3: per-lane binary traversal over the octant node copies.
template <bool kCount, int kStack, int kMode>
__device__ __forceinline__ void query(const TraceArgs& a, bool active, float3 o, float3 d, int skip, Hit& h,
                                      unsigned& nvis, unsigned& ntri, bool& ovf)
{
    if (kMode == 2) {
        closest_hit_packet<kCount, (kStack < 64 ? kStack : 64)>(a.nodes, tri_refs(a), active, o, d, skip, a.visit_limit, h,
                                                                nvis, ntri, ovf);
    } else if (active) {
        if (kMode == 1) closest_hit4<kCount, kStack>(a.nodes, tri_refs(a), o, d, skip, a.visit_limit, h, nvis, ntri, ovf);
        else if (kMode == 3)
            closest_hit_oct<kCount, kStack>(a.nodes, a.n_nodes, tri_refs(a), o, d, skip, a.visit_limit, h, nvis, ntri, ovf);
        else closest_hit<kCount, kStack>(a.nodes, tri_refs(a), o, d, skip, a.visit_limit, h, nvis, ntri, ovf);
    }
    if (active) key_closest(tri_refs(a), o, d, h);
}

// ---------------------------------------------------------------- silhouette mask
// Ray (i, j) of an aspect travels along k through the aperture point
// u = u0 + i ds, v = v0 + j ds (u, v along H and V; u0, v0 those of P0). It can
// only hit a triangle whose projection contains (u, v); the FP32 ray origin,
// the intersection slack (2^-12 of the determinant) and the FP32 projection
// below all stay within the margin of 0.01 cell + 2^-10 of the triangle's
// projected extent + 2^-18 of its distance from P0 (in cells). One thread
// projects one triangle for one aspect and ORs its cells into the tile words.
// A triangle whose widened box spans more than 2^16 cells sets the aspect's
// "all rays" flag (word total_tiles + aspect) instead.
// The grid cells (i0..i1, j0..j1) of aspect A whose rays the FP32 test could
// accept on triangle (a: v0, b: e1, c: e2); false if none.
// ids = 1 / sqrt(A.dA), the inverse grid spacing (FP32, set with the aspect table)
__device__ __forceinline__ float cell_scale(const AngleDev& A) { return A.ids; }

// The triangle's vertices projected onto the aspect's grid (in cells from P0),
// their ranges and their largest distance from P0 (in cells)
struct TriProj {
    float u[3], v[3], umin, umax, vmin, vmax, mag;
};

__device__ __forceinline__ void tri_project(const AngleDev& A, float ids, float4 a, float4 b, float4 c, TriProj& pr)
{
    const float px[3] = {a.x, a.x + b.x, a.x + c.x}, py[3] = {a.y, a.y + b.y, a.y + c.y},
                pz[3] = {a.z, a.z + b.z, a.z + c.z};
    pr.umin = FLT_MAX;
    pr.umax = -FLT_MAX;
    pr.vmin = FLT_MAX;
    pr.vmax = -FLT_MAX;
    pr.mag = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float dx = px[k] - A.p0[0], dy = py[k] - A.p0[1], dz = pz[k] - A.p0[2];
        const float u = (dx * A.hhat[0] + dy * A.hhat[1] + dz * A.hhat[2]) * ids;
        const float v = (dx * A.vhat[0] + dy * A.vhat[1] + dz * A.vhat[2]) * ids;
        pr.u[k] = u;
        pr.v[k] = v;
        pr.umin = fminf(pr.umin, u);
        pr.umax = fmaxf(pr.umax, u);
        pr.vmin = fminf(pr.vmin, v);
        pr.vmax = fmaxf(pr.vmax, v);
        pr.mag = fmaxf(pr.mag, (fabsf(dx) + fabsf(dy) + fabsf(dz)) * ids);
    }
}

__device__ __forceinline__ bool tri_cells_p(const AngleDev& A, const TriProj& pr, int& i0, int& i1, int& j0, int& j1)
{
    const float umin = pr.umin, umax = pr.umax, vmin = pr.vmin, vmax = pr.vmax;
    if (!(umin <= umax) || !(vmin <= vmax)) return false;  // NaN vertices: no ray can hit it
    const float m = 0.01f + (umax - umin + vmax - vmin) * (1.f / 1024.f) + pr.mag * (1.f / 262144.f);
    const float fi0 = ceilf(umin - m), fi1 = floorf(umax + m), fj0 = ceilf(vmin - m), fj1 = floorf(vmax + m);
    if (fi1 < 0.f || fj1 < 0.f || fi0 > (float)(A.nu - 1) || fj0 > (float)(A.nv - 1)) return false;
    i0 = max(0, (int)fi0);
    i1 = min(A.nu - 1, (int)fi1);
    j0 = max(0, (int)fj0);
    j1 = min(A.nv - 1, (int)fj1);
    return true;
}

__device__ __forceinline__ bool tri_cells(const AngleDev& A, float ids, float4 a, float4 b, float4 c, int& i0, int& i1,
                                          int& j0, int& j1)
{
    TriProj pr;
    tri_project(A, ids, a, b, c, pr);
    return tri_cells_p(A, pr, i0, i1, j0, j1);
}

// The projected triangle as three edge half-planes in the cell coordinates of
// an item's range (origin at its first cell i0, j0): cell (i, j) passes when
// nx (i - i0) + ny (j - j0) + c <= 0 for every edge. Each half-plane is moved
// outward by the margin m of tri_cells (the vertices' and ray origins' FP32
// errors) plus 0.002 cells (the local shift) and 1e-5 of the range per unit of
// |n| (the evaluation), so every cell of the conservative range whose ray the
// exact test can accept passes: the moved half-planes contain the projection
// widened by m in u and v. A projection of (nearly) zero area keeps every
// cell of the range.
struct CellEdges {
    float nx[3], ny[3], c[3];
};

__device__ __forceinline__ void tri_cell_edges_p(const TriProj& pr, int i0, int i1, int j0, int j1, CellEdges& E)
{
    float u[3], v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        u[k] = pr.u[k] - (float)i0;
        v[k] = pr.v[k] - (float)j0;
    }
    const float m =
        0.01f + (pr.umax - pr.umin + pr.vmax - pr.vmin) * (1.f / 1024.f) + pr.mag * (1.f / 262144.f) + 0.002f;
    const float a2 = (u[1] - u[0]) * (v[2] - v[0]) - (v[1] - v[0]) * (u[2] - u[0]);
    const float sg = a2 > 0.f ? 1.f : -1.f;
    const bool flat = !(fabsf(a2) > 1e-2f);
    const float ext = 1e-5f * (float)(i1 - i0 + j1 - j0 + 2);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int k1 = k == 2 ? 0 : k + 1;
        // outward normal of edge k -> k1 (counter-clockwise after the sign sg)
        const float nx = sg * (v[k1] - v[k]), ny = -sg * (u[k1] - u[k]);
        const float w = (fabsf(nx) + fabsf(ny)) * (m + ext);
        E.nx[k] = flat ? 0.f : nx;
        E.ny[k] = flat ? 0.f : ny;
        E.c[k] = flat ? -1.f : -(nx * u[k] + ny * v[k]) - w;
    }
}

__device__ __forceinline__ void tri_cell_edges(const AngleDev& A, float ids, float4 a, float4 b, float4 c, int i0,
                                               int i1, int j0, int j1, CellEdges& E)
{
    TriProj pr;
    tri_project(A, ids, a, b, c, pr);
    tri_cell_edges_p(pr, i0, i1, j0, j1, E);
}

__device__ __forceinline__ bool cell_inside(const CellEdges& E, int di, int dj)
{
    const float x = (float)di, y = (float)dj;
    return fmaf(E.nx[0], x, fmaf(E.ny[0], y, E.c[0])) <= 0.f && fmaf(E.nx[1], x, fmaf(E.ny[1], y, E.c[1])) <= 0.f &&
           fmaf(E.nx[2], x, fmaf(E.ny[2], y, E.c[2])) <= 0.f;
}

__global__ void __launch_bounds__(256) k_silhouette(const float4* __restrict__ tris, int n_tri,
                                                    const AngleDev* __restrict__ angles,
                                                    const long long* __restrict__ ray_off, int n_angles,
                                                    long long total_tiles, unsigned* cover)
{
    for (int ang = blockIdx.y; ang < n_angles; ang += gridDim.y) {
        const AngleDev& A = angles[ang];
        const int tw = A.tw_log2, W = 1 << tw, H = 32 >> tw;
        const float ids = cell_scale(A);
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tri; t += gridDim.x * blockDim.x) {
            const float4 a = __ldg(tris + 3 * (size_t)t), b = __ldg(tris + 3 * (size_t)t + 1),
                         c = __ldg(tris + 3 * (size_t)t + 2);
            int i0, i1, j0, j1;
            if (!tri_cells(A, ids, a, b, c, i0, i1, j0, j1)) continue;
            if ((long long)(i1 - i0 + 1) * (j1 - j0 + 1) > 65536) {
                atomicOr(cover + total_tiles + ang, 1u);
                continue;
            }
            const long long base = ray_off[ang];
            for (int j = j0; j <= j1; ++j) {
                const int bv = j / H, jl = j - bv * H;
                for (int i = i0; i <= i1;) {
                    const int bu = i >> tw, ie = min(i1, (bu << tw) + W - 1);
                    // bits (jl W + i % W) .. (jl W + ie % W) of tile (bv nbu + bu)
                    const int lo = jl * W + (i & (W - 1)), hi = jl * W + (ie & (W - 1));
                    const unsigned bits = (hi - lo == 31) ? 0xFFFFFFFFu : (((1u << (hi - lo + 1)) - 1u) << lo);
                    atomicOr(cover + ((base >> 5) + (long long)bv * A.nbu + bu), bits);
                    i = ie + 1;
                }
            }
        }
    }
}

// origin of primary ray (i, j) of aspect A (Eq. L1-L3 grid), in FP32
__device__ __forceinline__ float3 primary_origin(const AngleDev& A, int i, int j)
{
    const float fi = (float)i, fj = (float)j;
    return make_float3(__fadd_rn(__fadd_rn(A.p0[0], __fmul_rn(fi, A.du[0])), __fmul_rn(fj, A.dv[0])),
                       __fadd_rn(__fadd_rn(A.p0[1], __fmul_rn(fi, A.du[1])), __fmul_rn(fj, A.dv[1])),
                       __fadd_rn(__fadd_rn(A.p0[2], __fmul_rn(fi, A.du[2])), __fmul_rn(fj, A.dv[2])));
}

// ---------------------------------------------------------------- primary hits by rasterisation
// All primary rays of an aspect are parallel, so the closest hit of every ray
// can be found triangle by triangle: the FP32 test of a triangle runs for every
// grid ray in its conservative cell range (the silhouette range, which
// contains every ray the test accepts), and each ray keeps the smallest key
// (t bits << 32 | original index) by a 64-bit atomic minimum. t > 0, so the
// key order is (t, index): the closest hit and the tie rule of the traversal,
// whose t is <= FLT_MAX. A triangle spanning more than kRasterMaxCells cells
// flags its aspect instead, whose primary rays then traverse the tree.

// An aspect's ray grid held in registers for the cell loops: the loops' atomics
// could alias the aspect table as far as the compiler knows, so fields read
// through it would be loaded again after every atomic.
struct RasterGrid {
    float3 p0, du, dv, d;
    int nbu, tw;
};

__device__ __forceinline__ RasterGrid raster_grid(const AngleDev& A)
{
    RasterGrid G;
    G.p0 = make_float3(A.p0[0], A.p0[1], A.p0[2]);
    G.du = make_float3(A.du[0], A.du[1], A.du[2]);
    G.dv = make_float3(A.dv[0], A.dv[1], A.dv[2]);
    G.d = make_float3(A.dir[0], A.dir[1], A.dir[2]);
    G.nbu = A.nbu;
    G.tw = A.tw_log2;
    return G;
}

// the origin of grid ray (i, j): primary_origin's operations in its order
__device__ __forceinline__ float3 grid_origin(const RasterGrid& G, int i, int j)
{
    const float fi = (float)i, fj = (float)j;
    return make_float3(__fadd_rn(__fadd_rn(G.p0.x, __fmul_rn(fi, G.du.x)), __fmul_rn(fj, G.dv.x)),
                       __fadd_rn(__fadd_rn(G.p0.y, __fmul_rn(fi, G.du.y)), __fmul_rn(fj, G.dv.y)),
                       __fadd_rn(__fadd_rn(G.p0.z, __fmul_rn(fi, G.du.z)), __fmul_rn(fj, G.dv.z)));
}

// A triangle seen by the parallel rays of an aspect (direction d): the cross
// products of the triangle test depend on d and the triangle only, so with
// S = o - v0, U = S.(d x e2), V = S.(e1 x d) and T = S.(e1 x e2) (the same triple
// products) are three dot products per ray. Their error bounds are those of
// tri_filter (each below 8 u sum|S_i| of the absolute cross products).
struct RasterTri {
    float3 v0, p, p2, nn;  // vertex 0, d x e2, e1 x d, e1 x e2
    float det, bd;         // e1 . (d x e2) and its error bound (-1: degenerate, no hits)
    float bU, bV, bT;      // error bounds of U, V and T for every cell of the range
};

// The per-cell bounds 8.1 u |S|.(|d| x |e2|), 8.1 u |S|.(|e1| x |d|) and
// 9.1 u |S|.(|e1| x |e2|) taken once for the cell range i0..i1, j0..j1: each
// |S_c| is at most its largest value at the range's corner rays (|o - v0| is
// convex in (i, j) for the exact grid points) plus 8 u of the largest |o_c|
// (the FP32 rounding of the ray origins and of S).
__device__ __forceinline__ RasterTri raster_tri(const RasterGrid& G, float4 P, float4 B, float4 C, int i0, int i1,
                                                int j0, int j1)
{
    RasterTri R;
    const float3 e1 = make_float3(B.x, B.y, B.z), e2 = make_float3(C.x, C.y, C.z), d = G.d;
    R.v0 = make_float3(P.x, P.y, P.z);
    R.p = cross_s(d, e2);
    R.p2 = cross_s(e1, d);
    R.nn = cross_s(e1, e2);
    R.det = dot_s(e1, R.p);
    const float3 pa = cross_abs(d, e2);
    R.bd = B.w > 0.f ? 0x1.03p-21f * dot_s(abs3(e1), pa) : -1.f;
    float3 sm = make_float3(0.f, 0.f, 0.f), om = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float3 o = grid_origin(G, (c & 1) ? i1 : i0, (c & 2) ? j1 : j0);
        sm = make_float3(fmaxf(sm.x, fabsf(o.x - R.v0.x)), fmaxf(sm.y, fabsf(o.y - R.v0.y)),
                         fmaxf(sm.z, fabsf(o.z - R.v0.z)));
        om = make_float3(fmaxf(om.x, fabsf(o.x)), fmaxf(om.y, fabsf(o.y)), fmaxf(om.z, fabsf(o.z)));
    }
    const float g = 8.f * kU;
    sm = make_float3(__fmaf_rn(g, om.x + fabsf(R.v0.x), sm.x), __fmaf_rn(g, om.y + fabsf(R.v0.y), sm.y),
                     __fmaf_rn(g, om.z + fabsf(R.v0.z), sm.z));
    R.bU = 0x1.03p-21f * dot_s(sm, pa);
    R.bV = 0x1.03p-21f * dot_s(sm, cross_abs(e1, d));
    R.bT = 0x1.23p-21f * dot_s(sm, cross_abs(e1, e2));
    return R;
}

__device__ __forceinline__ void raster_cell(const RasterGrid& G, const TraceArgs& a, const RasterTri& R,
                                            const PlaneKey& K, int k, unsigned orig, int i, int j,
                                            unsigned long long* vrow, int count)
{
    const float3 o = grid_origin(G, i, j);
    const float3 s = make_float3(__fsub_rn(o.x, R.v0.x), __fsub_rn(o.y, R.v0.y), __fsub_rn(o.z, R.v0.z));
    float tc, et;
    // V = S.(e1 x d) and T = S.(e1 x e2) are the triple products of tri_filter, with the same bounds
    const int f = filter_core(dot_s(s, R.p), dot_s(s, R.p2), dot_s(s, R.nn), R.det, R.bU, R.bV, R.bd, R.bT, tc, et);
    if (f == 0) return;
    if (f >= 2) {
        const int r = tri_refine(a.tris, a.tri_v12, k, o, G.d, f, tc);
        if (count) count_open(a.stats, r);
        if (!(r & 1)) return;
    }
    const float th = plane_key_t(K, R.v0, o, tc);
    if (th >= 0.f && th <= FLT_MAX) {
        const int tw = G.tw, sh = 5 - tw;  // tile of W = 2^tw by H = 2^sh rays
        const int bu = i >> tw, bv = j >> sh;
        const long long pidx = ((long long)(bv * G.nbu + bu) << 5) + ((j & ((1 << sh) - 1)) << tw) + (i & ((1 << tw) - 1));
        atomicMin(vrow + pidx, ((unsigned long long)__float_as_uint(th) << 32) | orig);
    }
}

// A triangle of the flattened rasterisation and everything its cells need,
// one per lane in shared memory as 13 16-byte words (a stride of 52 words: the
// 16-byte accesses of 8 lanes to different triangles fall in distinct banks,
// and lanes reading one triangle's fields share a broadcast):
//   g0 = (p0.x, p0.y, p0.z, du.x)   g1 = (du.y, du.z, dv.x, dv.y)   g2 = (dv.z, v0.x, v0.y, v0.z)
//   r0 = (p.x, p.y, p.z, p2.x)      r1 = (p2.y, p2.z, nn.x, nn.y)   r2 = (nn.z, det, bd, bU)
//   r3 = (bV, bT, n.x, n.y)         r4 = (n.z, dh, dl, rd)           [plane key K]
//   e0 = (nx0, ny0, c0, nx1)        e1 = (ny1, c1, nx2, ny2)         e2 = (c2, 1 / w, tnear, ray_off)
//   m0 = (i0, j0, w, orig)          m1 = (aspect, triangle, nbu, tw)
// tnear: below the smallest stored distance any cell of the range can give
// this triangle (a cell whose ray already holds a closer hit is skipped).
struct __align__(16) RasterItem {
    float4 g0, g1, g2, r0, r1, r2, r3, r4, e0, e1, e2;
    int4 m0, m1;
};
static_assert(sizeof(RasterItem) == 52 * 4, "RasterItem layout");
constexpr int kRasterWarps = 8;    // warps of a k_raster block
constexpr int kRasterFlat = 512;   // cells of a triangle the warps flatten; larger ones go to k_raster_big
constexpr size_t kRasterSmem = sizeof(RasterItem) * 32 * kRasterWarps;

// Items q = aspect * n_tri + triangle, one per lane in grid-stride order
// (aspect-major: neighbouring lanes take neighbouring triangles of one
// aspect). Each lane projects its triangle and, for a range of at most
// kRasterFlat cells, writes the triangle's constants to shared memory; the
// warp then walks the (triangle, cell) pairs of its 32 triangles, lane l taking
// pairs l, l + 32, ..., so every lane works until the warp's cells run out. A
// triangle with a larger range is appended to the list `big` (warp-aggregated)
// for k_raster_big. Each cell passes the edge pretest before the triangle test.
__global__ void __launch_bounds__(256, 4) k_raster(const TraceArgs a, int n_tri, unsigned long long* vis, unsigned* full,
                                                   int count)
{
    extern __shared__ RasterItem s_items[];
    __shared__ int s_off[kRasterWarps][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    RasterItem* my = s_items + warp * 32;
    int* off = s_off[warp];
    const unsigned long long n_items = (unsigned long long)a.n_angles * (unsigned long long)n_tri;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long q0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    int ang = (int)(q0 / (unsigned long long)n_tri), t = (int)(q0 % (unsigned long long)n_tri);
    const int step_a = (int)(stride / (unsigned long long)n_tri), step_t = (int)(stride % (unsigned long long)n_tri);
    unsigned long long ntri = 0;
    // the rounds depend on the warp only: every lane reaches the ballots and shuffles
    for (unsigned long long base = q0 - lane; base < n_items; base += stride) {
        bool want_big = false;
        int4 rng = make_int4(0, 0, 0, 0);
        int nc = 0;
        if (base + lane < n_items) {
            const AngleDev& A = a.angles[ang];
            const float4* tp = a.tris + 3 * (size_t)t;
            const float4 P = __ldg(tp), B = __ldg(tp + 1), C = __ldg(tp + 2);
            int i0, i1, j0, j1;
            TriProj pr;
            tri_project(A, cell_scale(A), P, B, C, pr);
            if (tri_cells_p(A, pr, i0, i1, j0, j1)) {
                const long long ncell = (long long)(i1 - i0 + 1) * (j1 - j0 + 1);
                if (ncell > kRasterMaxCells || A.nu > 65535 || A.nv > 65535) {
                    atomicOr(full + ang, 1u);
                    atomicOr(full + a.n_angles, 1u);  // some aspect of the chunk traverses
                } else if (ncell > kRasterFlat) {
                    want_big = true;
                    rng = make_int4(t, ang, i0 | (j0 << 16), (i1 - i0) | ((j1 - j0) << 16));
                } else {
                    // each group of constants goes to shared memory as soon as it is formed
                    RasterItem& it = my[lane];
                    float c2;
                    {
                        CellEdges E;
                        tri_cell_edges_p(pr, i0, i1, j0, j1, E);
                        it.e0 = make_float4(E.nx[0], E.ny[0], E.c[0], E.nx[1]);
                        it.e1 = make_float4(E.ny[1], E.c[1], E.nx[2], E.ny[2]);
                        c2 = E.c[2];
                    }
                    const RasterGrid G = raster_grid(A);
                    float bd;
                    {
                        const RasterTri R = raster_tri(G, P, B, C, i0, i1, j0, j1);
                        it.g2 = make_float4(G.dv.z, R.v0.x, R.v0.y, R.v0.z);
                        it.r0 = make_float4(R.p.x, R.p.y, R.p.z, R.p2.x);
                        it.r1 = make_float4(R.p2.y, R.p2.z, R.nn.x, R.nn.y);
                        it.r2 = make_float4(R.nn.z, R.det, R.bd, R.bU);
                        it.r3 = make_float4(R.bV, R.bT, 0.f, 0.f);
                        bd = R.bd;
                    }
                    if (bd >= 0.f) {
                        const PlaneKey K = plane_key(a.tri_nrm, t, G.d);
                        it.r3.z = K.n.x;
                        it.r3.w = K.n.y;
                        it.r4 = make_float4(K.n.z, K.dh, K.dl, K.rd);
                        // distances along d of the vertices from the grid plane (the ray origins lie in it to
                        // within micrometres); the stored distance of any hit on the triangle is at least their
                        // minimum less the key's plane slack (0.08 bUV / |d.n|, as in key_of), 1e-4 of it and 1 mm
                        const float3 q0 = make_float3(P.x - G.p0.x, P.y - G.p0.y, P.z - G.p0.z);
                        const float z0 = dot_s(q0, G.d), z1 = z0 + dot_s(make_float3(B.x, B.y, B.z), G.d),
                                    z2 = z0 + dot_s(make_float3(C.x, C.y, C.z), G.d);
                        const float zm = fminf(z0, fminf(z1, z2));
                        const float slack = K.dh != 0.f ? 0.32f * B.w / fabsf(K.dh) : FLT_MAX;
                        const float tnear = zm - (1e-4f * fabsf(zm) + 1e-3f + slack);
                        it.e2 = make_float4(c2, 1.f / (float)(i1 - i0 + 1), isfinite(tnear) ? tnear : -FLT_MAX,
                                            __int_as_float((int)a.ray_off[ang]));
                        it.g0 = make_float4(G.p0.x, G.p0.y, G.p0.z, G.du.x);
                        it.g1 = make_float4(G.du.y, G.du.z, G.dv.x, G.dv.y);
                        it.m0 = make_int4(i0, j0, i1 - i0 + 1, __float_as_int(P.w));
                        it.m1 = make_int4(ang, t, G.nbu, G.tw);
                        nc = (int)ncell;
                    }
                }
            }
        }
        const unsigned m = __ballot_sync(kFull, want_big);
        if (m) {
            unsigned slot = 0;
            if (lane == __ffs(m) - 1) slot = atomicAdd(a.big_ctr, (unsigned)__popc(m));
            slot = __shfl_sync(kFull, slot, __ffs(m) - 1) + __popc(m & ((1u << lane) - 1u));
            if (want_big) {
                if (slot < a.big_cap) {
                    a.big[slot] = rng;
                } else {  // no room: this aspect's primary rays traverse
                    atomicOr(full + rng.y, 1u);
                    atomicOr(full + a.n_angles, 1u);
                }
            }
        }
        // inclusive scan of the cell counts: off[k] = first pair of lane k's triangle
        int incl = nc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        off[lane + 1] = incl;
        if (lane == 0) off[0] = 0;
        __syncwarp();
        const int total = __shfl_sync(kFull, incl, 31);
        int k = 0;
        for (int c = lane; c < total; c += 32) {
            while (off[k + 1] <= c) ++k;
            const RasterItem& it = my[k];
            const int loc = c - off[k];
            const int4 m0 = it.m0;
            const float4 e0 = it.e0, e1 = it.e1, e2 = it.e2;
            // (loc + 0.5) / w is at least 0.5 / w from an integer and loc, w <= 512: the FP32 product floors exactly
            const int dj = __float2int_rz(((float)loc + 0.5f) * e2.y), di = loc - dj * m0.z;
            {
                const float x = (float)di, y = (float)dj;
                if (!(fmaf(e0.x, x, fmaf(e0.y, y, e0.z)) <= 0.f && fmaf(e0.w, x, fmaf(e1.x, y, e1.y)) <= 0.f &&
                      fmaf(e1.z, x, fmaf(e1.w, y, e2.x)) <= 0.f))
                    continue;
            }
            const int i = m0.x + di, j = m0.y + dj;
            const int4 m1 = it.m1;
            const int tw = m1.w, sh = 5 - tw;  // tile of W = 2^tw by H = 2^sh rays
            const long long pidx = (long long)__float_as_int(e2.w) + ((long long)((j >> sh) * m1.z + (i >> tw)) << 5) +
                                   ((j & ((1 << sh) - 1)) << tw) + (i & ((1 << tw) - 1));
            // the ray's closest hit so far (keys only decrease; a stale value is larger): nearer than any
            // distance this triangle can give, the cell is decided
            if (__uint_as_float((unsigned)(__ldcg(vis + pidx) >> 32)) < e2.z) continue;
            ++ntri;
            const float4 g0 = it.g0, g1 = it.g1, g2 = it.g2;
            const float fi = (float)i, fj = (float)j;
            const float3 o = make_float3(__fadd_rn(__fadd_rn(g0.x, __fmul_rn(fi, g0.w)), __fmul_rn(fj, g1.z)),
                                         __fadd_rn(__fadd_rn(g0.y, __fmul_rn(fi, g1.x)), __fmul_rn(fj, g1.w)),
                                         __fadd_rn(__fadd_rn(g0.z, __fmul_rn(fi, g1.y)), __fmul_rn(fj, g2.x)));
            const float3 v0 = make_float3(g2.y, g2.z, g2.w);
            const float3 sv = make_float3(__fsub_rn(o.x, v0.x), __fsub_rn(o.y, v0.y), __fsub_rn(o.z, v0.z));
            const float4 r0 = it.r0, r1 = it.r1, r2 = it.r2, r3 = it.r3;
            float tc, et;
            const int f = filter_core(dot_s(sv, make_float3(r0.x, r0.y, r0.z)), dot_s(sv, make_float3(r0.w, r1.x, r1.y)),
                                      dot_s(sv, make_float3(r1.z, r1.w, r2.x)), r2.y, r2.w, r3.x, r2.z, r3.y, tc, et);
            if (f == 0) continue;
            if (f >= 2) {
                const AngleDev& A = a.angles[m1.x];
                const int r = tri_refine(a.tris, a.tri_v12, m1.y, o, make_float3(A.dir[0], A.dir[1], A.dir[2]), f, tc);
                if (count) count_open(a.stats, r);
                if (!(r & 1)) continue;
            }
            const float4 r4 = it.r4;
            PlaneKey K;
            K.n = make_float3(r3.z, r3.w, r4.x);
            K.dh = r4.y;
            K.dl = r4.z;
            K.rd = r4.w;
            const float th = plane_key_t(K, v0, o, tc);
            if (th >= 0.f && th <= FLT_MAX)
                atomicMin(vis + pidx, ((unsigned long long)__float_as_uint(th) << 32) | (unsigned)m0.w);
        }
        __syncwarp();  // the next round rewrites my[] and off[]
        t += step_t;
        ang += step_a;
        if (t >= n_tri) {
            t -= n_tri;
            ++ang;
        }
    }
    if (count) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ntri += __shfl_xor_sync(kFull, ntri, o);
        if (lane == 0 && ntri) {
            atomicAdd(a.stats + kStatTris, ntri);
            atomicAdd(a.stats + kStatRaster, ntri);
        }
    }
}

// The listed large triangles, warp w taking entries w, w + warps, ... (every
// warp has hundreds of entries, so the few very large triangles average out),
// their cells 32 at a time.
__global__ void __launch_bounds__(256, 3) k_raster_big(const TraceArgs a, unsigned long long* vis, int count)
{
    const int lane = threadIdx.x & 31;
    const unsigned n_big = min(a.big_ctr[0], a.big_cap);
    const unsigned nw = (gridDim.x * blockDim.x) >> 5;
    unsigned long long ntri = 0;
    for (unsigned it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < n_big; it += nw) {
        const int4 b = a.big[it];
        const int td = b.x, ad = b.y;
        const int i0 = b.z & 0xFFFF, j0 = (unsigned)b.z >> 16, w = (b.w & 0xFFFF) + 1, h = ((unsigned)b.w >> 16) + 1;
        const int i1 = i0 + w - 1, j1 = j0 + h - 1;
        const AngleDev& A = a.angles[ad];
        const RasterGrid G = raster_grid(A);
        const float4* tp = a.tris + 3 * (size_t)td;
        const float4 P = __ldg(tp), B = __ldg(tp + 1), C = __ldg(tp + 2);
        const RasterTri R = raster_tri(G, P, B, C, i0, i1, j0, j1);
        if (!(R.bd >= 0.f)) continue;  // warp-uniform
        const unsigned orig = (unsigned)__float_as_int(P.w);
        unsigned long long* vrow = vis + a.ray_off[ad];
        const PlaneKey K = plane_key(a.tri_nrm, td, G.d);
        CellEdges E;
        tri_cell_edges(A, cell_scale(A), P, B, C, i0, i1, j0, j1, E);
        const int ncell = w * h;
        // cell c = (c / w, c % w) from (j0, i0); steps of 32 cells: sj rows and si columns
        const int sj = 32 / w, si = 32 - sj * w, l0 = lane / w;
        int i = i0 + (lane - l0 * w), j = j0 + l0;
        for (int cidx = lane; cidx < ncell; cidx += 32) {
            if (cell_inside(E, i - i0, j - j0)) {
                raster_cell(G, a, R, K, td, orig, i, j, vrow, count);
                ++ntri;
            }
            i += si;
            j += sj;
            if (i > i1) {
                i -= w;
                ++j;
            }
        }
    }
    if (count) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ntri += __shfl_xor_sync(kFull, ntri, o);
        if (lane == 0 && ntri) {
            atomicAdd(a.stats + kStatTris, ntri);
            atomicAdd(a.stats + kStatRaster, ntri);
        }
    }
}

// contiguous tile range [t0, t1) of warp gw of nw over n_tiles tiles
__device__ __forceinline__ void warp_tiles(long long n_tiles, long long gw, long long nw, long long& t0, long long& t1)
{
    const long long per = (n_tiles + nw - 1) / nw;
    t0 = gw * per;
    t1 = t0 + per < n_tiles ? t0 + per : n_tiles;
}

// valid bits of the rasterised primary rays (0 for the tiles of flagged
// aspects, which traverse); each warp a contiguous range of tiles
__global__ void __launch_bounds__(256) k_vis_mask(const TraceArgs a, const unsigned long long* __restrict__ vis,
                                                  const unsigned* __restrict__ full, unsigned* mask)
{
    const int lane = threadIdx.x & 31;
    long long t0, t1;
    warp_tiles(a.total_rays >> 5, ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
               ((long long)gridDim.x * blockDim.x) >> 5, t0, t1);
    if (t0 >= t1) return;  // warp-uniform
    const bool any_full = full[a.n_angles] != 0;
    int ang = 0;
    if (any_full) {
        if (lane == 0) ang = find_angle(a.ray_off, a.n_angles, t0 << 5);
        ang = __shfl_sync(kFull, ang, 0);
    }
#pragma unroll 4
    for (long long tile = t0; tile < t1; ++tile) {
        unsigned m = __ballot_sync(kFull, vis[(tile << 5) + lane] != ~0ull);
        if (any_full) {
            while (a.ray_off[ang + 1] <= (tile << 5)) ++ang;
            if (full[ang]) m = 0;
        }
        if (lane == 0) mask[tile] = m;
    }
}

// ---------------------------------------------------------------- pass 0: primary rays
// state of a primary ray before its first hit: receive basis field, path
// term k.o0 (two-float), no bounce yet
__device__ __forceinline__ void start_ray(const AngleDev& A, Ray& r)
{
    r.ev = make_float3(A.vhat[0], A.vhat[1], A.vhat[2]);
    tf_dot(A.dir, r.o, r.lacc_hi, r.lacc_lo);
    r.cos0 = 0.f;
    r.nb = 0;
    r.last = -1;
}

template <bool kCount, int kStack, int kMode>
__global__ void __launch_bounds__(kTraceThreads, 4) k_primary(const TraceArgs a)
{
    // with rasterised hits this kernel only traverses for flagged aspects
    if (a.vis && !a.vis_full[a.n_angles]) return;
    const int lane = threadIdx.x & 31;
    unsigned nq = 0, nvis = 0, ntri = 0;
    bool ovf = false;
    while (true) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.work, 32ull);
        base = __shfl_sync(kFull, base, 0);
        if ((long long)base >= a.total_rays) break;
        int ang = 0;
        if (lane == 0) ang = find_angle(a.ray_off, a.n_angles, (long long)base);
        ang = __shfl_sync(kFull, ang, 0);
        if (a.vis && !a.vis_full[ang]) continue;  // warp-uniform; k_primary_vis takes this tile
        const AngleDev& A = a.angles[ang];
        const int local = (int)((long long)base + lane - a.ray_off[ang]);
        int i, j;
        tile_ij(A, local, i, j);
        bool active = i < A.nu && j < A.nv;
        if (a.cover)
            active = active && (((a.cover[base >> 5] >> lane) & 1u) || a.cover[(a.total_rays >> 5) + ang]);
        bool hit = false;
        Ray r;
        r.angle = ang;
        r.local = local;
        r.o = make_float3(0.f, 0.f, 0.f);
        r.d = make_float3(0.f, 0.f, 1.f);
        if (active) {
            r.o = primary_origin(A, i, j);
            r.d = make_float3(A.dir[0], A.dir[1], A.dir[2]);
        }
        Hit h;
        query<kCount, kStack, kMode>(a, active, r.o, r.d, -1, h, nvis, ntri, ovf);
        if (active) {
            ++nq;
            if (h.k >= 0) {
                start_ray(a.angles[ang], r);
                hit = true;
                apply_hit(A, a.tri_nrm, h, a.flags, r);
                record_hit(a, r, h);
            }
        }
        const unsigned m = __ballot_sync(kFull, hit);
        if (lane == 0) a.mask[base >> 5] = m;
        push(a, hit, r);
    }
    flush_stats<kCount>(a, nq, nvis, ntri, ovf);
}

// Primary pass of the rasterised aspects. The hit rays go to the queue slots
// given by the scan of the raster masks (no atomics). Without a hit list each
// ray reads its key and its state is written to its slot, the tiles assigned
// statically (every tile costs about the same). With a hit list only (ray,
// aspect) of each hit is written, from the mask words and slots alone.
template <bool kCount, bool kList>
__global__ void __launch_bounds__(kTraceThreads) k_primary_vis(const TraceArgs a)
{
    const int lane = threadIdx.x & 31;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gw = gtid >> 5, nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long n_tiles = a.total_rays >> 5;
    // one primary query per grid ray of every rasterised aspect
    unsigned nq = 0;
    for (long long ang = gtid; ang < a.n_angles; ang += (long long)gridDim.x * blockDim.x)
        if (!a.vis_full[ang]) nq += (unsigned)a.angles[ang].nu * (unsigned)a.angles[ang].nv;
    if (kList) {
        // 32 tiles per warp step: lane l loads the mask word and slot of tile t0 + l, then the warp
        // writes the list entries tile by tile (a set bit implies a rasterised aspect: k_vis_mask
        // clears the masks of flagged ones)
        long long t0 = gw << 5;
        int ang = 0;
        long long next = 0;
        if (t0 < n_tiles) {
            if (lane == 0) ang = find_angle(a.ray_off, a.n_angles, t0 << 5);
            ang = __shfl_sync(kFull, ang, 0);
            next = a.ray_off[ang + 1];
        }
        for (; t0 < n_tiles; t0 += nw << 5) {
            const long long t = t0 + lane;
            unsigned m = 0, slot = 0;
            if (t < n_tiles) {
                m = a.mask[t];
                if (m) slot = a.tile_base[t];
            }
            unsigned todo = __ballot_sync(kFull, m != 0u);
            while (todo) {
                const int k = __ffs(todo) - 1;
                todo &= todo - 1u;
                const unsigned mk = __shfl_sync(kFull, m, k), sk = __shfl_sync(kFull, slot, k);
                const long long base = (t0 + k) << 5;
                while (next <= base) next = a.ray_off[++ang + 1];  // the tiles of a warp only move forward
                if ((mk >> lane) & 1u)
                    a.hit_list[sk + __popc(mk & ((1u << lane) - 1u))] = make_uint2((unsigned)(base + lane), (unsigned)ang);
            }
        }
    } else {
        constexpr int kChunk = 4;  // tiles of a chunk; chunks interleaved over the warps (hits cluster in the grid)
        const long long n_chunks = (n_tiles + kChunk - 1) / kChunk;
        int ang = 0;
        if (gw < n_chunks) {
            if (lane == 0) ang = find_angle(a.ray_off, a.n_angles, (gw * kChunk) << 5);
            ang = __shfl_sync(kFull, ang, 0);
        }
        for (long long chunk = gw; chunk < n_chunks; chunk += nw) {
            for (long long tile = chunk * kChunk; tile < (chunk + 1) * kChunk && tile < n_tiles; ++tile) {
                const long long base = tile << 5;
                while (a.ray_off[ang + 1] <= base) ++ang;  // the tiles of a warp only move forward
                const unsigned vmask = a.mask[tile];        // k_vis_mask; 0 for a flagged aspect
                if (!((vmask >> lane) & 1u)) continue;
                const AngleDev& A = a.angles[ang];
                const int local = (int)(base + lane - a.ray_off[ang]);
                int i, j;
                tile_ij(A, local, i, j);
                const unsigned long long key = __ldcs(a.vis + base + lane);
                Hit h;
                h.t = __uint_as_float((unsigned)(key >> 32));
                h.orig = (int)(unsigned)key;
                h.k = __ldg(a.tri_pos + h.orig);
                Ray r;
                r.angle = ang;
                r.local = local;
                r.o = primary_origin(A, i, j);
                r.d = make_float3(A.dir[0], A.dir[1], A.dir[2]);
                start_ray(A, r);
                apply_hit(A, a.tri_nrm, h, a.flags, r);
                record_hit(a, r, h);
                store_state(a.q_out, a.tile_base[tile] + __popc(vmask & ((1u << lane) - 1u)), r);
            }
        }
    }
    flush_stats<kCount>(a, nq, 0u, 0u, false);
}

// ---------------------------------------------------------------- pass b >= 1: live rays
// State of rasterised primary hit (ray g of the chunk, aspect ang) after its
// first hit: the same steps as k_primary_vis.
__device__ __forceinline__ void primary_state(const TraceArgs& a, unsigned g, int ang, Ray& r)
{
    const AngleDev& A = a.angles[ang];
    const int local = (int)((long long)g - a.ray_off[ang]);
    int i, j;
    tile_ij(A, local, i, j);
    const unsigned long long key = __ldcs(a.vis + g);
    Hit h;
    h.t = __uint_as_float((unsigned)(key >> 32));
    h.orig = (int)(unsigned)key;
    h.k = __ldg(a.tri_pos + h.orig);
    r.angle = ang;
    r.local = local;
    r.o = primary_origin(A, i, j);
    r.d = make_float3(A.dir[0], A.dir[1], A.dir[2]);
    start_ray(A, r);
    apply_hit(A, a.tri_nrm, h, a.flags, r);
    record_hit(a, r, h);
}

// Origin, direction and triangle after the first hit of a rasterised primary
// ray (ray g of the chunk, aspect ang): the stored-state steps of apply_hit
// alone (hit point, orientation, reflection, offset origin).
__device__ __forceinline__ void primary_geom(const TraceArgs& a, unsigned g, int ang, float3& o, float3& d, int& last)
{
    const AngleDev& A = a.angles[ang];
    int i, j;
    tile_ij(A, (int)((long long)g - a.ray_off[ang]), i, j);
    const unsigned long long key = __ldcs(a.vis + g);
    const float t = __uint_as_float((unsigned)(key >> 32));
    const int k = __ldg(a.tri_pos + (int)(unsigned)key);
    const float3 o0 = primary_origin(A, i, j), d0 = make_float3(A.dir[0], A.dir[1], A.dir[2]);
    const float3 x = make_float3(__fmaf_rn(t, d0.x, o0.x), __fmaf_rn(t, d0.y, o0.y), __fmaf_rn(t, d0.z, o0.z));
    const float4 N4 = __ldg(a.tri_nrm + k);
    const float3 n = make_float3(N4.x, N4.y, N4.z);
    float dn, dnl;
    tf_dot3(d0, n, dn, dnl);
    const float3 nf = dn < 0.f ? n : make_float3(-n.x, -n.y, -n.z);
    const float m2 = -2.f * dn;
    d = make_float3(__fmaf_rn(m2, n.x, d0.x), __fmaf_rn(m2, n.y, d0.y), __fmaf_rn(m2, n.z, d0.z));
    o = make_float3(__fmaf_rn(A.eps, nf.x, x.x), __fmaf_rn(A.eps, nf.y, x.y), __fmaf_rn(A.eps, nf.z, x.z));
    last = k;
}

template <bool kCount, int kStack, int kMode, bool kBi = false, bool kList = false>
__global__ void __launch_bounds__(kTraceThreads, 4) k_bounce(const TraceArgs a)
{
    const int lane = threadIdx.x & 31;
    const unsigned n_in = *a.q_in_count;
    const unsigned n_list = kList ? *a.list_count : 0u;  // entries below n_list come from the hit list
    const bool escape_pass = a.bounce >= a.max_bounces;
    unsigned nq = 0, nvis = 0, ntri = 0, nhit = 0, nlist = 0;  // hits processed, hits rebuilt (counting runs)
    unsigned long long wvis = 0;  // counting runs: 32 x the warp's largest node visit count, per query
    bool ovf = false;
    while (true) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.work, 32ull);
        base = __shfl_sync(kFull, base, 0);
        if (base >= n_in) break;
        const unsigned idx = (unsigned)base + lane;
        bool again = false;
        Ray r;
        const bool active = idx < n_in;
        r.o = make_float3(0.f, 0.f, 0.f);
        r.d = make_float3(0.f, 0.f, 1.f);
        r.last = -1;
        const bool listed = kList && idx < n_list;
        uint2 e = make_uint2(0u, 0u);
        if (listed) {
            // only the geometry during the query; the full state after it
            e = a.hit_list[idx];
            primary_geom(a, e.x, (int)e.y, r.o, r.d, r.last);
            if (kCount) ++nlist;
        }
        // the pass's i-th entry, in the order of q_order when the rays were grouped by place
        const unsigned src = (a.q_order && active && !listed) ? __ldcs(a.q_order + idx) : idx;
        if (active && !listed) load_geom(a.q_in, src, r);
        Hit h;
        const unsigned nvis0 = nvis;
        query<kCount, kStack, kMode>(a, active, r.o, r.d, r.last, h, nvis, ntri, ovf);
        if (kCount) wvis += 32ull * __reduce_max_sync(kFull, nvis - nvis0);
        if (active) {
            if (listed) primary_state(a, e.x, (int)e.y, r);
            else load_payload(a.q_in, src, r);
            const AngleDev& A = a.angles[r.angle];
            ++nq;
            if (h.k < 0) {
                // escaped: its last hit radiates
                emit(a, r, kBi && A.bistatic && !rx_visible(a, A, r, nq, ovf));
            } else if (escape_pass) {
                emit(a, r, true);                      // still trapped after B_max: invalid
            } else {
                if (kCount) ++nhit;
                apply_hit(A, a.tri_nrm, h, a.flags, r);
                record_hit(a, r, h);
                if (r.nb < a.max_bounces || (a.flags & kFlagEscape)) again = true;
                else emit(a, r, kBi && A.bistatic && !rx_visible(a, A, r, nq, ovf));
            }
        }
        push(a, again, r);
    }
    flush_stats<kCount>(a, nq, nvis, ntri, ovf, nhit, nlist, (threadIdx.x & 31) == 0 ? wvis : 0ull);
}

// every ray of the queue writes its record (B_max = 1 without the escape check)
template <bool kBi>
__global__ void __launch_bounds__(kTraceThreads) k_emit_all(const TraceArgs a)
{
    const unsigned n_in = *a.q_in_count;
    unsigned nq = 0;
    bool ovf = false;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n_in; i += gridDim.x * blockDim.x) {
        Ray r;
        load_state(a.q_in, i, r);
        const AngleDev& A = a.angles[r.angle];
        emit(a, r, kBi && A.bistatic && !rx_visible(a, A, r, nq, ovf));
    }
    if (nq) atomicAdd(a.stats + kStatQueries, (unsigned long long)nq);
    if (ovf) atomicAdd(a.stats + kStatOverflow, 1ull);
}

// ---------------------------------------------------------------- pooled late passes
// The live rays that a chunk's early passes leave for the next pass go to a
// pool shared by the chunks (push above), so that the late passes run once over
// the rays of every chunk: a late pass holds few rays per chunk, and a launch
// over few rays leaves most of the GPU idle while its slowest rays finish.
// k_pool_append moves rays that a chunk kept because the pool was full into the
// pool once it has been traced (their aspect index shifted by angle_shift, 0
// for rays push already gave the trace's index).
__global__ void __launch_bounds__(256) k_pool_append(const RayState* __restrict__ src, const unsigned* src_count,
                                                     RayState* __restrict__ pool, const unsigned* pool_count,
                                                     unsigned cap, int angle_shift)
{
    const unsigned n = *src_count, at = *pool_count;
    if ((unsigned long long)at + n > cap) return;  // k_pool_commit raises the flag
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4* p = reinterpret_cast<const float4*>(src + i);
        float4* q = reinterpret_cast<float4*>(pool + at + i);
#pragma unroll
        for (int w = 0; w < 5; ++w) __stcs(q + w, __ldcs(p + w));
        int4 g = __ldcs(reinterpret_cast<const int4*>(p) + 5);
        g.x += angle_shift;
        __stcs(reinterpret_cast<int4*>(q) + 5, g);
    }
}

// Rays grouped by place before a pooled pass: the rays of one aspect that
// leave neighbouring triangles (the reordered triangles follow the tree's
// leaves) start close together, in similar directions, and share much of
// their traversal. A counting sort by bucket with atomic cursors; the order
// within a bucket varies between runs and changes no result, since every ray
// writes its record to the slot its primary ray reserved.
__device__ __forceinline__ unsigned ray_bucket(const RayState* __restrict__ q, unsigned i, int tri_shift,
                                               unsigned groups)
{
    const int4 g = __ldcs(reinterpret_cast<const int4*>(q + i) + 5);  // aspect, ray, triangle left, bounces
    return (unsigned)g.x * groups + ((unsigned)g.z >> tri_shift);
}

// Neighbouring queue entries mostly share a bucket (a warp's survivors are
// appended together), so the lanes of a warp that share one make a single
// atomic for all of them. The loops run whole warps (every lane reaches the
// match).
__global__ void __launch_bounds__(256) k_bucket_count(const RayState* __restrict__ q, const unsigned* count,
                                                      int tri_shift, unsigned groups, unsigned* counts)
{
    const unsigned n = *count;
    const int lane = threadIdx.x & 31;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned w = blockIdx.x * blockDim.x + threadIdx.x - lane; w < n; w += stride) {
        const unsigned i = w + lane;
        const unsigned b = i < n ? ray_bucket(q, i, tri_shift, groups) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(kFull, b);
        if (i < n && lane == __ffs(peers) - 1) atomicAdd(counts + b, (unsigned)__popc(peers));
    }
}

__global__ void __launch_bounds__(256) k_bucket_scatter(const RayState* __restrict__ q, const unsigned* count,
                                                        int tri_shift, unsigned groups, unsigned* cursor,
                                                        unsigned* order)
{
    const unsigned n = *count;
    const int lane = threadIdx.x & 31;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned w = blockIdx.x * blockDim.x + threadIdx.x - lane; w < n; w += stride) {
        const unsigned i = w + lane;
        const unsigned b = i < n ? ray_bucket(q, i, tri_shift, groups) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(kFull, b);
        const int leader = __ffs(peers) - 1;
        unsigned base = 0;
        if (i < n && lane == leader) base = atomicAdd(cursor + b, (unsigned)__popc(peers));
        base = __shfl_sync(kFull, base, leader);
        if (i < n) order[base + __popc(peers & ((1u << lane) - 1u))] = i;
    }
}

__global__ void k_pool_commit(const unsigned* src_count, unsigned* pool_count, unsigned cap, unsigned* flag)
{
    const unsigned n = *src_count, at = *pool_count;
    if ((unsigned long long)at + n > cap) *flag = 1u;
    else *pool_count = at + n;
}

__global__ void k_angle_offsets(const long long* ray_off, const unsigned* tile_base, const unsigned* total,
                                int n_angles, unsigned* rec_off)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_angles) rec_off[i] = tile_base[ray_off[i] >> 5];
    if (i == n_angles) rec_off[i] = *total;
}

}  // namespace

int trace_blocks_per_sm()
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bounce<false, 64, 0>, kTraceThreads, 0);
    return nb > 0 ? nb : 1;
}

template <int kStack, int kMode>
void launch_trace_s(const TraceArgs& a, int n_blocks, bool count_visits, cudaStream_t st)
{
    if (a.bounce == 0) {
        if (a.vis) {
            if (a.hit_list) {
                if (count_visits) k_primary_vis<true, true><<<n_blocks, kTraceThreads, 0, st>>>(a);
                else k_primary_vis<false, true><<<n_blocks, kTraceThreads, 0, st>>>(a);
            } else {
                if (count_visits) k_primary_vis<true, false><<<n_blocks, kTraceThreads, 0, st>>>(a);
                else k_primary_vis<false, false><<<n_blocks, kTraceThreads, 0, st>>>(a);
            }
        }
        if (count_visits) k_primary<true, kStack, kMode><<<n_blocks, kTraceThreads, 0, st>>>(a);
        else k_primary<false, kStack, kMode><<<n_blocks, kTraceThreads, 0, st>>>(a);
    } else if (a.bounce == 1 && a.hit_list) {
        if (count_visits) k_bounce<true, kStack, kMode, false, true><<<n_blocks, kTraceThreads, 0, st>>>(a);
        else k_bounce<false, kStack, kMode, false, true><<<n_blocks, kTraceThreads, 0, st>>>(a);
    } else {
        if (count_visits) k_bounce<true, kStack, kMode><<<n_blocks, kTraceThreads, 0, st>>>(a);
        else k_bounce<false, kStack, kMode><<<n_blocks, kTraceThreads, 0, st>>>(a);
    }
}

template <int kMode>
void launch_trace_m(const TraceArgs& a, int n_blocks, bool count_visits, int stack_depth, cudaStream_t st)
{
    if (stack_depth == 32) {
        launch_trace_s<32, kMode>(a, n_blocks, count_visits, st);
        return;
    }
    if constexpr (kMode != 2) {
        if (stack_depth == 128) {
            launch_trace_s<128, kMode>(a, n_blocks, count_visits, st);
            return;
        }
    }
    launch_trace_s<64, kMode>(a, n_blocks, count_visits, st);
}

cudaError_t launch_trace(const TraceArgs& a, int n_blocks, bool count_visits, int stack_depth, cudaStream_t st)
{
    if (a.bistatic && a.bounce > 0) {
        // bounce passes of chunks with a bistatic aspect: per-lane traversal, 64-entry stack, visibility tests
        if (a.wide) {
            if (count_visits) k_bounce<true, 64, 1, true><<<n_blocks, kTraceThreads, 0, st>>>(a);
            else k_bounce<false, 64, 1, true><<<n_blocks, kTraceThreads, 0, st>>>(a);
        } else if (a.octant) {
            if (count_visits) k_bounce<true, 64, 3, true><<<n_blocks, kTraceThreads, 0, st>>>(a);
            else k_bounce<false, 64, 3, true><<<n_blocks, kTraceThreads, 0, st>>>(a);
        } else {
            if (count_visits) k_bounce<true, 64, 0, true><<<n_blocks, kTraceThreads, 0, st>>>(a);
            else k_bounce<false, 64, 0, true><<<n_blocks, kTraceThreads, 0, st>>>(a);
        }
        return cudaGetLastError();
    }
    if (a.wide) launch_trace_m<1>(a, n_blocks, count_visits, stack_depth, st);
    else if (a.packet) launch_trace_m<2>(a, n_blocks, count_visits, stack_depth, st);
    else if (a.octant) launch_trace_m<3>(a, n_blocks, count_visits, stack_depth, st);
    else launch_trace_m<0>(a, n_blocks, count_visits, stack_depth, st);
    return cudaGetLastError();
}

cudaError_t launch_emit_all(const TraceArgs& a, int n_blocks, cudaStream_t st)
{
    if (a.bistatic) k_emit_all<true><<<n_blocks, kTraceThreads, 0, st>>>(a);
    else k_emit_all<false><<<n_blocks, kTraceThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_group_rays(const RayState* q, const unsigned* count, int tri_shift, unsigned groups,
                              unsigned* counts, long long n_buckets, unsigned* order, void* scratch, int n_blocks,
                              cudaStream_t st)
{
    k_bucket_count<<<n_blocks, 256, 0, st>>>(q, count, tri_shift, groups, counts);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = scan_exclusive_u32(counts, counts, n_buckets, false, nullptr, scratch, st);
    if (e != cudaSuccess) return e;
    k_bucket_scatter<<<n_blocks, 256, 0, st>>>(q, count, tri_shift, groups, counts, order);
    return cudaGetLastError();
}

cudaError_t launch_pool_append(const RayState* src, const unsigned* src_count, RayState* pool, unsigned* pool_count,
                               unsigned cap, int angle_shift, unsigned* flag, int n_blocks, cudaStream_t st)
{
    k_pool_append<<<n_blocks, 256, 0, st>>>(src, src_count, pool, pool_count, cap, angle_shift);
    k_pool_commit<<<1, 1, 0, st>>>(src_count, pool_count, cap, flag);
    return cudaGetLastError();
}

cudaError_t launch_silhouette(const TraceArgs& a, int n_tri, unsigned* cover, cudaStream_t st)
{
    if (a.n_angles <= 0 || n_tri <= 0) return cudaSuccess;
    const int bx = (int)std::min<long long>((n_tri + 255) / 256, 64);
    const int by = std::min(a.n_angles, 4096);
    k_silhouette<<<dim3(bx, by), 256, 0, st>>>(a.tris, n_tri, a.angles, a.ray_off, a.n_angles, a.total_rays >> 5,
                                               cover);
    return cudaGetLastError();
}

cudaError_t launch_raster(const TraceArgs& a, int n_tri, unsigned long long* vis, unsigned* full, bool count,
                          int n_blocks, void* scan_scratch, cudaStream_t st)
{
    if (a.n_angles <= 0 || n_tri <= 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(vis, 0xFF, sizeof(unsigned long long) * (size_t)a.total_rays, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(full, 0, sizeof(unsigned) * (size_t)(a.n_angles + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.big_ctr, 0, sizeof(unsigned) * 2, st);
    if (e != cudaSuccess) return e;
    static int smem_set[64] = {0};  // per device: k_raster's dynamic shared memory above 48 KB allowed
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!smem_set[dev]) {
        e = cudaFuncSetAttribute(k_raster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRasterSmem);
        if (e != cudaSuccess) return e;
        smem_set[dev] = 1;
    }
    const long long need = ((long long)a.n_angles * n_tri + 255) / 256;
    k_raster<<<(int)std::max(1ll, std::min<long long>(need, n_blocks)), 32 * kRasterWarps, kRasterSmem, st>>>(
        a, n_tri, vis, full, count ? 1 : 0);
    k_raster_big<<<n_blocks, 256, 0, st>>>(a, vis, count ? 1 : 0);
    const long long n_tiles = a.total_rays >> 5;
    k_vis_mask<<<(int)std::max(1ll, std::min<long long>((n_tiles + 7) / 8, n_blocks)), 256, 0, st>>>(a, vis, full,
                                                                                                     a.mask);
    e = cudaGetLastError();
    // queue slots of the rasterised hits; the traversing rays append after them
    if (e == cudaSuccess)
        e = scan_popc(a.mask, const_cast<unsigned*>(a.tile_base), n_tiles, a.list_count, scan_scratch, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(a.q_out_count, a.list_count, sizeof(unsigned), cudaMemcpyDeviceToDevice, st);
    return e;
}

cudaError_t launch_angle_offsets(const long long* ray_off, const unsigned* tile_base, const unsigned* total,
                                 int n_angles, unsigned* rec_off, cudaStream_t st)
{
    k_angle_offsets<<<(n_angles + 1 + 255) / 256, 256, 0, st>>>(ray_off, tile_base, total, n_angles, rec_off);
    return cudaGetLastError();
}

}  // namespace sbr
