// sbr_internal.h -- device data layouts and launcher declarations shared by the
// translation units of libsbr (not part of the public ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sbr {

// ---------------------------------------------------------------- BVH layout
// A BVH node stores the boxes of both children, so one 64-byte fetch gives the
// traversal everything it needs to test and order the two children:
//   n0 = (L.lo.x, L.hi.x, L.lo.y, L.hi.y)
//   n1 = (R.lo.x, R.hi.x, R.lo.y, R.hi.y)
//   n2 = (L.lo.z, L.hi.z, R.lo.z, R.hi.z)
//   n3 = (ref L, ref R, 0, 0)   (int bits)
// ref >= 0 is an internal node index; ref < 0 is a leaf whose triangles are the
// contiguous range [first, first + count) of the reordered triangle array:
//   ref = 0x80000000 | first << 4 | (count - 1),  count in 1..16.
// kEmptyRef marks a missing child (its box is empty: lo > hi).
constexpr int kLeafMax = 16;
constexpr int kEmptyRef = (int)0xFFFFFFFF;

__host__ __device__ inline int leaf_ref(int first, int count)
{
    return (int)(0x80000000u | ((unsigned)first << 4) | (unsigned)(count - 1));
}
__host__ __device__ inline int leaf_first(int ref) { return (int)(((unsigned)ref & 0x7FFFFFFFu) >> 4); }
__host__ __device__ inline int leaf_count(int ref) { return (int)((unsigned)ref & 15u) + 1; }

// A triangle is 3 float4 (48 bytes): (v0, original index as int bits), (e1, bUV),
// (e2, bD) with e1 = v1 - v0, e2 = v2 - v0 rounded to FP32 and the constants of
// the FP32 filter's error bounds, u = 2^-24 and L = max(|e1|_1, |e2|_1):
//   bUV = 24 u L (1 + 2^-10),  bD = 14 u L^2 (1 + 2^-10)
// (all zero for a degenerate triangle: it takes no hits). Beside the records,
// at the same position: tri_nrm = (n32, 0), the FP32 rounding of the FP64 unit
// normal, read for the hit point, the reflection and the hit distance; and
// tri_v12 = (v1, 0), (v2, 0), the exact vertices, read only when the filter
// leaves a decision open and it is taken again in FP64.

// ---------------------------------------------------------------- per-aspect data
struct AngleDev {            // 192 bytes
    float p0[3], du[3], dv[3], dir[3];  // FP32 ray grid: o(i, j) = (p0 + i du) + j dv
    float rhat[3], vhat[3], hhat[3];    // radar direction, V (theta_hat), H (phi_hat)
    float dA, eps;                      // tube area ds^2, origin offset after a hit
    int nu, nv;
    long long ray_off;                  // first ray of this aspect in the chunk, multiple of 32
    int nbu;                            // ray tiles per aperture row: ceil(nu / tile width)
    int tw_log2;                        // tile width 2^tw_log2 (height 32 / width): one warp per tile
    int bistatic;                       // 1: receiver below differs from the transmitter (visibility test)
    int pad;
    float rxr[3], rxv[3], rxh[3];       // receiver direction and its V, H basis (= rhat, vhat, hhat monostatic)
    float rxdir[3];                     // -rxr in FP32 (= dir monostatic): the path term of the receiver
    float ids;                          // 1 / sqrt(dA) in FP32: grid cells per metre (rasterisation)
    float pad2[3];
};
static_assert(sizeof(AngleDev) == 192, "AngleDev layout");

// live ray between bounces (96 bytes, three 32-byte sectors)
struct __align__(16) RayState {
    float ox, oy, oz, dx;
    float dy, dz, evx, evy;
    float evz, lacc_hi, lacc_lo, cos0;  // E of the V transmit case; path so far (two-float)
    float c0, c1, c2, c3;               // candidate tube coefficients HH, VV, HV, VH at the last hit
    float cs, lc_hi, lc_lo, nfs;        // candidate scalar coefficient, candidate path L (two-float), side of the
                                        // last hit's normal facing the incoming ray (+1 / -1)
    int angle, local, last, nb;         // aspect (chunk-local), processing index (8x4 tiles), last sorted triangle, bounces
};
static_assert(sizeof(RayState) == 96, "RayState layout");

// dense valid-hit record consumed by the PO reduction (32 bytes)
struct __align__(16) Record {
    float c[5];         // HH, VV, HV, VH (vector form) and the scalar form coefficient
    float l_hi, l_lo;   // path L as an unevaluated FP32 sum
    int ray;            // ray id j*nu + i within its aspect
};
static_assert(sizeof(Record) == 32, "Record layout");

// stats counters on the device (unsigned long long each)
enum { kStatQueries = 0, kStatNodes = 1, kStatTris = 2, kStatOverflow = 3, kStatRaster = 4, kStatHits = 5, kStatListed = 6,
       kStatOpen = 7, kStatFp64 = 8, kStatWarpNodes = 9, kStatCount = 10 };

// ---------------------------------------------------------------- launchers
// All launchers enqueue on `st` and return the launch error (cudaSuccess if none).

// 4-wide BVH (collapsed from the binary one): node k is 8 float4 (128 bytes)
//   f0 = lo.x, f1 = hi.x, f2 = lo.y, f3 = hi.y, f4 = lo.z, f5 = hi.z  (children 0..3 in x, y, z, w)
//   f6 = (ref 0, ref 1, ref 2, ref 3)  (int bits, same encoding as above; kEmptyRef for a missing child,
//         whose box is empty: lo = +FLT_MAX, hi = -FLT_MAX)
//   f7 = 0
// Node 0 is the root. Each child box is the box of a binary node or leaf, so
// the 4-wide tree tests exactly the boxes the binary tree would.
constexpr int kNode4Float4 = 8;
// Octant copies of the binary nodes: copy o (bit 0: x, bit 1: y, bit 2: z set
// when the ray's direction is negative on that axis) stores for both children
// the near and far slab of each axis already chosen (near = lo on a positive
// axis, hi on a negative one):
//   f0 = (L.near.x, L.near.y, L.near.z, R.near.x)
//   f1 = (R.near.y, R.near.z, L.far.x, L.far.y)
//   f2 = (L.far.z, R.far.x, R.far.y, R.far.z)
//   f3 = (ref L, ref R, 0, 0)
// at octant_nodes[(o * n_nodes + k) * 4 ..]. An empty child box (lo = +FLT_MAX,
// hi = -FLT_MAX) has near > far on every axis, so it is never entered.
cudaError_t build_octant_nodes(const float4* nodes, long long n_nodes, float4* out, cudaStream_t st);
// Collapse the binary node array (root 0) into nodes4 (room for max(n_tri - 1, 1) nodes).
// queue_a / queue_b: int2 [max(n_tri - 1, 1)]; counters: int [4]. A tree of at most 16384 binary
// nodes is collapsed by one block in one launch; a larger one synchronises once per level.
// *n_nodes4 receives the node count.
cudaError_t bvh4_collapse(const float4* nodes2, long long n_nodes2, float4* nodes4, int2* queue_a, int2* queue_b,
                          int* counters, int* n_nodes4, cudaStream_t st);

struct BvhBuild {
    // inputs
    const float* xyz;
    const int* tri;
    long long n_vert, n_tri;
    int leaf_max;
    float c_t, c_i;
    int builder;  // 0: Karras LBVH with SAH refit; 1: PLOC clustering (synchronises per round)
    int radius;   // PLOC search radius (0: 16)
    // outputs (allocated by the caller: nodes [max(n_tri-1,1)*4] float4, tris [n_tri*3] float4)
    float4* nodes;
    float4* tris;
    float4* tri_nrm;  // [n_tri] (n32, 0) per reordered triangle
    float4* tri_v12;  // [2 n_tri] (v1, 0), (v2, 0) per reordered triangle
    int* tri_pos;     // [n_tri]: position in tris of each original triangle index
    float* bbox_out;  // device float[6] scene box of the vertices
    int* err_flag;    // device int: bit 1 a triangle index out of range, bit 2 a non-finite coordinate,
                      // bit 4 the clustering did not converge
    int* n_nodes_out; // device int: reachable nodes, numbered 0.. in depth-first order
    // scratch (caller-owned)
    void* scratch;
    size_t scratch_bytes;
};
size_t bvh_scratch_bytes(long long n_tri);
cudaError_t bvh_build(const BvhBuild& b, cudaStream_t st);

struct TraceArgs {
    const float4* nodes;          // binary nodes, or 4-wide nodes when wide = 1
    int wide;
    int packet;                   // 1: warp-cooperative traversal of the binary tree
    int bistatic;                 // 1: some aspect of the chunk has a bistatic receiver (visibility tests)
    int octant;                   // 1: nodes are the octant copies of the binary nodes (n_nodes per copy)
    long long n_nodes;
    const float4* tris;
    const float4* tri_nrm;        // [n_tri] FP32 unit normals (reordered like tris)
    const float4* tri_v12;        // [2 n_tri] exact v1, v2 (reordered like tris)
    const AngleDev* angles;
    const long long* ray_off;     // [n_angles + 1] chunk-relative, multiples of 32
    int n_angles;
    int max_bounces;
    int bounce;                   // index of this pass (0 = primary rays)
    int flags;
    int visit_limit;              // upper bound of node + leaf visits of one query (2 n_tri + 64)
    long long total_rays;         // primary: padded ray count of the chunk
    const RayState* q_in;
    const unsigned* q_order;      // optional: entry i of the pass is q_in[q_order[i]] (rays grouped by place)
    const unsigned* q_in_count;
    RayState* q_out;
    unsigned* q_out_count;
    unsigned* mask;               // [total_rays / 32] valid bits of primary rays
    const unsigned* cover;        // optional [total_rays / 32 + n_angles] silhouette bits (0 = the ray surely
                                  // misses) and per-aspect all-rays flags
    const unsigned* tile_base;    // [total_rays / 32] exclusive prefix of popcount(mask)
    Record* rec;                  // dense records of this chunk (already offset to the chunk)
    const long long* rec_of;      // pooled late passes (else null): per aspect, the first record of its
                                  // chunk; rec is then the record buffer itself
    RayState* pool;               // optional: the pass appends the rays that go on to this ray pool (their
    unsigned* pool_count;         // aspect index + angle_shift) while it holds fewer than pool_cap; those
    unsigned pool_cap;            // that find it full go to q_out
    int angle_shift;
    unsigned long long* work;     // work counter (zeroed before each pass)
    unsigned long long* stats;    // [kStatCount]
    int* hit_tri;                 // optional [total_rays][max_bounces] (RECORD_HITS)
    float* hit_t;                 // optional [total_rays][max_bounces]
    int* hit_nb;                  // optional [total_rays]
    const unsigned long long* vis; // optional (primary pass) [total_rays] closest-hit keys from k_raster
    const unsigned* vis_full;     // with vis: [n_angles + 1] 1 = the aspect's primary rays traverse the tree;
                                  // [n_angles]: 1 if any aspect does
    const int* tri_pos;           // with vis: [n_tri] position in tris of each original triangle index
    unsigned* list_count;         // with vis: device count of the rasterised primary hits
    int4* big;                    // with vis: triangles of more than 32 cells, (triangle, aspect, i0 | j0 << 16,
                                  // (i1 - i0) | (j1 - j0) << 16), tested by warps after the per-thread pass
    unsigned* big_ctr;            // with vis: [2] entries appended, (unused)
    unsigned big_cap;             // with vis: capacity of big (an aspect whose entry does not fit traverses)
    uint2* hit_list;              // optional (rasterised hits, a bounce pass follows): the primary pass
                                  // lists (ray, aspect) of each rasterised hit here instead of storing
                                  // its state, and bounce pass 1 rebuilds the state from the list
};
int trace_blocks_per_sm();
// stack_depth: 32, 64 or 128 entries of the traversal stack (other values: 64;
// the warp-cooperative traversal uses at most 64)
cudaError_t launch_trace(const TraceArgs& a, int n_blocks, bool count_visits, int stack_depth, cudaStream_t st);
cudaError_t launch_emit_all(const TraceArgs& a, int n_blocks, cudaStream_t st);
// Append the *src_count live rays of src to the pool at *pool_count (their
// aspect index shifted by angle_shift), then advance *pool_count; when they do
// not fit under cap nothing is copied and *flag becomes 1.
// Group the *count rays of q by (aspect, triangle left >> tri_shift): bucket
// b = aspect * groups + (triangle >> tri_shift) of n_buckets; counts
// (n_buckets + 1 words, zeroed by the caller) becomes the buckets' starts, and
// order[i] the position in q of the i-th ray in bucket order (within a bucket
// in no particular order). scratch: scan_scratch_bytes(n_buckets + 1).
cudaError_t launch_group_rays(const RayState* q, const unsigned* count, int tri_shift, unsigned groups,
                              unsigned* counts, long long n_buckets, unsigned* order, void* scratch, int n_blocks,
                              cudaStream_t st);
cudaError_t launch_pool_append(const RayState* src, const unsigned* src_count, RayState* pool, unsigned* pool_count,
                               unsigned cap, int angle_shift, unsigned* flag, int n_blocks, cudaStream_t st);
// Silhouette mask of the aspects of a chunk (a.angles, a.ray_off, a.n_angles):
// sets cover bit (processing layout) of every grid ray whose (u, v) lies in
// the conservatively widened projected box of some triangle, or the aspect's
// all-rays flag (word a.total_rays / 32 + aspect) for a triangle too large to
// rasterise. cover must be zeroed first ([a.total_rays / 32 + a.n_angles] words).
cudaError_t launch_silhouette(const TraceArgs& a, int n_tri, unsigned* cover, cudaStream_t st);
// Primary closest hits by rasterisation (aspects a.angles, a.ray_off, a.n_angles
// of a chunk of a.total_rays rays): vis[g] becomes the smallest key
// (FP32 t bits << 32 | original triangle index) over the triangles whose FP32
// test accepts primary ray g, or ~0 for none; full[aspect] = 1 and
// full[n_angles] = 1 when a triangle covers more than kRasterMaxCells cells of
// that aspect (its rays then traverse the tree). Clears vis and full itself.
// Then sets a.mask to the valid bits of the rasterised rays, a.tile_base to
// their exclusive scan and *a.q_out_count to their number: the primary pass
// stores those rays at fixed queue slots and appends the traversing ones after
// them.
constexpr long long kRasterMaxCells = 1 << 14;
cudaError_t launch_raster(const TraceArgs& a, int n_tri, unsigned long long* vis, unsigned* full, bool count,
                          int n_blocks, void* scan_scratch, cudaStream_t st);

// exclusive scan of in[i] (or popcount(in[i])) -> out[i]; total written to *total
size_t scan_scratch_bytes(long long n);
cudaError_t scan_exclusive_u32(const unsigned* in, unsigned* out, long long n, bool popc, unsigned* total,
                               void* scratch, cudaStream_t st);
cudaError_t scan_popc(const unsigned* mask, unsigned* tile_base, long long n, unsigned* total, void* scratch,
                      cudaStream_t st);
cudaError_t launch_angle_offsets(const long long* ray_off, const unsigned* tile_base, const unsigned* total,
                                 int n_angles, unsigned* rec_off, cudaStream_t st);

struct PoItem {
    int angle;        // aspect index within the call
    int count;        // records in this item (at most kPoItem)
    long long first;  // first record
    int f0, nf;       // frequencies [f0, f0 + nf) of the frequency table
    long long part;   // first FP64 partial of this item: nf x n_pol x (re, im)
};
static_assert(sizeof(PoItem) == 32, "PoItem layout");
// per-aspect view of the items and of the output rows
struct PoAngle {
    int item_begin, item_end;  // items of this aspect
    int f0, nf;                // its frequencies in the frequency table
    long long out_row;         // first output row: row out_row + q holds frequency f0 + q
    long long part;            // first partial of its items (device-built work lists)
};
static_assert(sizeof(PoAngle) == 32, "PoAngle layout");
struct PoArgs {
    const Record* rec;
    const PoItem* items;
    int n_items;
    const int* n_items_dev;  // when set, the item count is read here (device-built work lists)
    int item_records;        // records per item: 512, 1024 or 2048 (kPoItemRecords when 0)
    const float4* freq;   // [n_freq] (kappa_hi, kappa_lo, k, 0), kappa = f / c0 cycles per metre
    const double* kfreq;  // [n_freq] k in FP64 (FP64 phase mode)
    int n_freq;           // entries of the frequency table
    int pol_sel[4];       // selected polarisation indices (0 HH, 1 VV, 2 HV, 3 VH)
    int n_pol;
    int scalar;           // 1: paper scalar form
    int phase_mode;       // 0 compensated, 1 FP32, 2 FP64
    double* partial;      // FP64 partials, item i at items[i].part
    int* err = nullptr;   // optional device flag: set when a bounded wait of the staged kernel gave up (the
                          // item's partials are then NaN); with it, single-frequency sums use that kernel
};
// n_blocks > 0: persistent grid of that many blocks looping over the items
cudaError_t launch_po(const PoArgs& a, cudaStream_t st, int n_blocks = 0);
// Device-built PO work list of one traced chunk: aspect a owns the records
// [recoff[a], recoff[a + 1]) of the chunk, cut into items of item_records.
// Fills angles[a].item_begin / item_end / part (f0, nf, out_row are inputs),
// items[] and *n_items; *valid = recoff[n_angles] (may be null).
constexpr int kPoItemRecords = 1024;
cudaError_t launch_po_items(const unsigned* recoff, PoAngle* angles, int n_angles, int n_pol, int item_records,
                            PoItem* items, int* n_items, long long* valid, cudaStream_t st);
// the work list from host-built aspect tables: 64-bit record offsets (n_angles + 1) and PoAngle rows
// whose item ranges and partial offsets are set
cudaError_t launch_po_items_fill(const long long* recoff, const PoAngle* angles, int n_angles, int n_pol,
                                 int item_records, PoItem* items, cudaStream_t st);
// E[row][n_pol][2] and rcs[row][n_pol] for every aspect's rows (fixed-order FP64 sums of the partials)
cudaError_t launch_po_final(const double* partial, const PoItem* items, const PoAngle* angles, int n_angles,
                            const double* kfreq, int n_pol, double* E, double* rcs, cudaStream_t st);

// ---------------------------------------------------------------- tensor-core GEMM (surrogate)
// C = A B^T, A [M x K] and B [N x K] BF16 with K contiguous; M, N multiples of
// 128 and K a multiple of 64. The epilogue is fused:
enum { kEpiF32 = 0, kEpiBiasGelu = 1, kEpiGeluGrad = 2 };
struct GemmEpi {
    int mode;                 // kEpi*
    int M;                    // rows of C
    float* c_f32;             // kEpiF32: C; kEpiBiasGelu: z = acc + bias, or null where no backward pass reads it
                              // (row stride ldc)
    int ldc;
    __nv_bfloat16* out_bf16;  // kEpiBiasGelu: gelu(z); kEpiGeluGrad: acc * gelu'(z)  (row stride ldo)
    int ldo;
    const float* bias;        // kEpiBiasGelu: [N]
    const float* z;           // kEpiGeluGrad: pre-activation [M x N] (row stride ldz)
    int ldz;
};
bool gemm_shape_ok(int M, int N, int K);
cudaError_t gemm_bf16_tn(const void* A, int lda, const void* B, int ldb, int M, int N, int K, const GemmEpi& ep,
                         int* err, cudaStream_t st);

}  // namespace sbr
