// sbr_api.cu -- host runtime behind the C ABI declared in include/sbr.h:
// context and stream ownership, device buffers, per-aspect ray frames
// (Eq. L1-L3), the chunked trace driver (Algorithm 2 as a wavefront of
// persistent passes) and the PO integration driver (Eq. po_sum).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <string>
#include <vector>

#include "sbr.h"
#include "sbr_internal.h"

using namespace sbr;

namespace {

constexpr double kC0 = 299792458.0;
constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxBounces = 128;

std::string g_create_error;

}  // namespace

namespace sbr {
// error message of a context-free call, returned by sbr_last_error(NULL)
void set_static_error(const char* msg) { g_create_error = msg; }
}  // namespace sbr

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes)
    {
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t want = std::max(bytes, (size_t)256);
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) cap = want;
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <class T>
    T* as() const { return (T*)p; }
};

struct AngleHost {
    sbr_ray_grid grid;
    int tw;               // ray tile width log2 used for this trace
    bool bistatic = false;
    double rx_az = 0.0, rx_el = 0.0;  // receiver of a bistatic aspect (degrees)
    long long ray_begin;  // first ray (padded layout) over the whole trace
    long long rec_begin, rec_count;
};

struct BatchPlan;
void free_plan(BatchPlan* p);

}  // namespace

struct sbr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int n_sms = 0;
    sbr_tuning tune;  // launch and layout parameters (sbr_set_tuning / sbr_autotune)
    std::string err;
    // mesh
    long long n_vert = 0, n_tri = 0;
    DevBuf xyz, tri;
    float bbox[6] = {0, 0, 0, 0, 0, 0};
    bool has_mesh = false, has_bvh = false;
    // BVH
    DevBuf nodes, tris, bvh_scratch, bbox_dev, err_dev;
    DevBuf nodes4;  // 4-wide collapse of the binary tree
    int n_nodes4 = 0;
    DevBuf nodes_oct;  // octant copies of the binary nodes (built on first use)
    long long n_nodes = 0, oct_gen = -1;
    // trace
    DevBuf angles, rayoff, mask, tilebase, scan_scr, recoff, q0, q1, ctr64, ctr32, stats, rec, cover;
    DevBuf hit_tri, hit_t, hit_nb;
    DevBuf tripos, vis, visfull;  // position of each original triangle; raster keys and per-aspect flags
    DevBuf rbig, rbigctr;         // large triangles of a rasterised chunk and their two counters
    long long rbig_cap = 0;
    DevBuf hitlist;               // (ray, aspect) of the rasterised primary hits, read by bounce pass 1
    // pooled late passes of sbr_trace: the live rays the chunks leave for pass kPoolPass, the trace's aspect
    // table and ray offsets, each aspect's first record, the pool's counters and work counters
    DevBuf pool, angall, rayoffall, recofall, poolctr, poolwork;
    DevBuf poolgroup;  // bucket counts, grouped order and scan scratch of the pooled passes' rays
    unsigned* pool_host = nullptr;  // pinned copy of the pool's count and flag
    long long rec_total = 0;
    int max_bounces = 0, trace_flags = 0;
    bool has_trace = false;
    std::vector<AngleHost> ang;
    // PO
    DevBuf items, itemoff, recbeg, freq, kfreq, partial, E, rcs;
    // pinned staging
    void* host_stage = nullptr;
    size_t host_stage_cap = 0;
    size_t stage_off = 0;  // first free byte of host_stage
    cudaEvent_t stage_ev = nullptr;  // recorded after the last enqueued copy that touches host_stage
    std::vector<cudaEvent_t> evpool; // pass timing events (SBR_TRACE_TIME_PASSES)
    // asynchronous batches (sbr_submit_batch)
    long long mesh_gen = 0;  // bumped whenever the BVH buffers change
    BatchPlan* plan = nullptr;
    bool plan_pending = false;
};

namespace {

int fail(sbr_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

int cuda_fail(sbr_ctx* c, cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(c, SBR_ERR_OOM, "%s: out of device memory", what);
    }
    return fail(c, SBR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

// A region of the pinned staging buffer for the caller's host-to-device or
// device-to-host copies. Regions are handed out one after another, so a new one
// never overlaps a region that an enqueued copy may still use; only when the
// buffer is full does the host wait (for stage_ev, which every caller records
// after its copies) and start again at the front. The caller must be done with
// the host side of earlier regions by its next call.
void* stage(sbr_ctx* c, size_t bytes)
{
    bytes = (bytes + 255) & ~(size_t)255;
    if (c->host_stage && c->stage_off + bytes <= c->host_stage_cap) {
        void* p = (char*)c->host_stage + c->stage_off;
        c->stage_off += bytes;
        return p;
    }
    if (c->stage_ev) cudaEventSynchronize(c->stage_ev);  // earlier async copies may still use the buffer
    c->stage_off = 0;
    if (bytes > c->host_stage_cap) {
        if (c->host_stage) {
            cudaStreamSynchronize(c->stream);
            cudaFreeHost(c->host_stage);
        }
        c->host_stage = nullptr;
        c->host_stage_cap = 0;
        size_t want = std::max(bytes, (size_t)(4 << 20));
        if (cudaMallocHost(&c->host_stage, want) != cudaSuccess) return nullptr;
        c->host_stage_cap = want;
    }
    c->stage_off = bytes;
    return c->host_stage;
}

// Per-aspect grid (Eq. L1-L3) in FP64, rounded once to FP32 where the device uses it.
// Arithmetic order is part of the ray-grid convention (bit-identical rays on
// every implementation of it); this file is built without FP contraction.
void make_grid(const float* bbox, double az_deg, double el_deg, double ds, double eta, const sbr_trace_opts* opt,
               sbr_ray_grid* g)
{
    memset(g, 0, sizeof(*g));
    const double a = az_deg * (kPi / 180.0), e = el_deg * (kPi / 180.0);
    const double ca = cos(a), sa = sin(a), ce = cos(e), se = sin(e);
    g->rhat[0] = ce * ca;
    g->rhat[1] = ce * sa;
    g->rhat[2] = se;
    for (int k = 0; k < 3; ++k) g->khat[k] = -g->rhat[k];
    g->vhat[0] = se * ca;
    g->vhat[1] = se * sa;
    g->vhat[2] = -ce;
    g->hhat[0] = -sa;
    g->hhat[1] = ca;
    g->hhat[2] = 0.0;
    double lo[3], hi[3], mid[3], s2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        lo[k] = (double)bbox[k];
        hi[k] = (double)bbox[3 + k];
        mid[k] = 0.5 * (lo[k] + hi[k]);
        s2 += (hi[k] - lo[k]) * (hi[k] - lo[k]);
    }
    const double diag = sqrt(s2);
    const double D = 0.5 * diag + 1.0;
    double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    for (int m = 0; m < 8; ++m) {
        const double p[3] = {(m & 1) ? hi[0] : lo[0], (m & 2) ? hi[1] : lo[1], (m & 4) ? hi[2] : lo[2]};
        const double pu = p[0] * g->hhat[0] + p[1] * g->hhat[1] + p[2] * g->hhat[2];
        const double pv = p[0] * g->vhat[0] + p[1] * g->vhat[1] + p[2] * g->vhat[2];
        umin = std::min(umin, pu);
        umax = std::max(umax, pu);
        vmin = std::min(vmin, pv);
        vmax = std::max(vmax, pv);
    }
    g->lu = umax - umin;
    g->lv = vmax - vmin;
    const double window = opt ? opt->window_m : 0.0;
    double xu, xv;
    if (window > 0.0) {
        xu = window / ds;
        xv = xu;
    } else {
        xu = (1.0 + eta) * g->lu / ds;
        xv = (1.0 + eta) * g->lv / ds;
    }
    g->nu = std::max<int64_t>(1, (int64_t)ceil(xu - 1e-9));
    g->nv = std::max<int64_t>(1, (int64_t)ceil(xv - 1e-9));
    g->spacing = ds;
    g->eps = 1e-5 * diag;
    const double offu = opt ? opt->offset_u : 0.0, offv = opt ? opt->offset_v : 0.0;
    const double au = (0.5 - 0.5 * (double)g->nu + offu) * ds;
    const double av = (0.5 - 0.5 * (double)g->nv + offv) * ds;
    for (int k = 0; k < 3; ++k) {
        g->p0[k] = (float)(((mid[k] - D * g->khat[k]) + au * g->hhat[k]) + av * g->vhat[k]);
        g->du[k] = (float)(ds * g->hhat[k]);
        g->dv[k] = (float)(ds * g->vhat[k]);
        g->dir[k] = (float)g->khat[k];
    }
}

// rx: (az, el) of a bistatic receiver in degrees, or null (receiver = transmitter)
AngleDev to_dev(const sbr_ray_grid& g, long long ray_off, int tw, const double* rx = nullptr)
{
    AngleDev d;
    memset(&d, 0, sizeof(d));
    for (int k = 0; k < 3; ++k) {
        d.p0[k] = g.p0[k];
        d.du[k] = g.du[k];
        d.dv[k] = g.dv[k];
        d.dir[k] = g.dir[k];
        d.rhat[k] = (float)g.rhat[k];
        d.vhat[k] = (float)g.vhat[k];
        d.hhat[k] = (float)g.hhat[k];
    }
    d.dA = (float)(g.spacing * g.spacing);
    d.ids = 1.f / sqrtf(d.dA);
    d.eps = (float)g.eps;
    d.nu = (int)g.nu;
    d.nv = (int)g.nv;
    d.nbu = (int)((g.nu + (1 << tw) - 1) >> tw);
    d.tw_log2 = tw;
    if (rx) {
        // same axis convention as the transmitter (make_grid)
        const double a = rx[0] * (kPi / 180.0), e = rx[1] * (kPi / 180.0);
        const double ca = cos(a), sa = sin(a), ce = cos(e), se = sin(e);
        const double rr[3] = {ce * ca, ce * sa, se}, vv[3] = {se * ca, se * sa, -ce}, hh[3] = {-sa, ca, 0.0};
        for (int k = 0; k < 3; ++k) {
            d.rxr[k] = (float)rr[k];
            d.rxv[k] = (float)vv[k];
            d.rxh[k] = (float)hh[k];
            d.rxdir[k] = (float)(-rr[k]);
        }
        d.bistatic = 1;
    } else {
        for (int k = 0; k < 3; ++k) {
            d.rxr[k] = d.rhat[k];
            d.rxv[k] = d.vhat[k];
            d.rxh[k] = d.hhat[k];
            d.rxdir[k] = d.dir[k];
        }
        d.bistatic = 0;
    }
    d.ray_off = ray_off;
    return d;
}

// rays an aspect occupies in the processing layout: whole tiles of 2^tw x 32 / 2^tw
// entries of the rasterisation's list of large triangles for a chunk of `rays` primary rays (an aspect whose
// large triangles do not fit traverses instead)
long long raster_big_cap(long long rays)
{
    return std::min<long long>(std::max<long long>(1ll << 16, rays / 4), 1ll << 30);
}

long long tiled_rays(const sbr_ray_grid& g, int tw)
{
    const long long th = 32 >> tw;
    return ((g.nu + (1ll << tw) - 1) >> tw) * ((g.nv + th - 1) / th) * 32;
}

int log2i(int v)
{
    int k = 0;
    while ((1 << (k + 1)) <= v) ++k;
    return k;
}

bool tuning_ok(const sbr_tuning& t)
{
    const bool tile = t.tile_w >= 1 && t.tile_w <= 32 && (t.tile_w & (t.tile_w - 1)) == 0;
    const bool trav = (t.packet == 0 || (t.packet == 1 && t.bvh_width == 2 && t.stack_depth <= 64)) &&
                      (t.silhouette == 0 || t.silhouette == 1) &&
                      (t.octant == 0 || (t.octant == 1 && t.bvh_width == 2 && t.packet == 0)) &&
                      (t.raster == 0 || t.raster == 1);
    return tile && trav && (t.bvh_width == 2 || t.bvh_width == 4) && t.blocks_per_sm >= 1 && t.blocks_per_sm <= 4 &&
           (t.stack_depth == 32 || t.stack_depth == 64 || t.stack_depth == 128) && t.chunk_rays_log2 >= 20 &&
           t.chunk_rays_log2 <= 29 && (t.po_item == 512 || t.po_item == 1024 || t.po_item == 2048);
}

}  // namespace

extern "C" {

int sbr_version(void) { return SBR_VERSION_MAJOR * 100 + SBR_VERSION_MINOR; }

const char* sbr_last_error(const sbr_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

double sbr_spacing_for(double f_max_hz, double rays_per_lambda)
{
    if (!(f_max_hz > 0.0) || !(rays_per_lambda > 0.0)) return -1.0;
    return kC0 / (f_max_hz * rays_per_lambda);
}

int sbr_create(sbr_ctx** out, int device, void* cuda_stream)
{
    if (!out) {
        g_create_error = "sbr_create: null output pointer";
        return SBR_ERR_ARG;
    }
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        g_create_error = std::string("sbr_create: no CUDA device (") + cudaGetErrorString(e) + ")";
        return SBR_ERR_NODEV;
    }
    if (device < 0 || device >= n) {
        g_create_error = "sbr_create: device index out of range";
        return SBR_ERR_ARG;
    }
    e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        g_create_error = std::string("sbr_create: cudaSetDevice: ") + cudaGetErrorString(e);
        return SBR_ERR_CUDA;
    }
    sbr_ctx* c = new sbr_ctx();
    c->device = device;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            g_create_error = std::string("sbr_create: stream: ") + cudaGetErrorString(e);
            delete c;
            return SBR_ERR_CUDA;
        }
        c->own_stream = true;
    }
    cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, device);
    e = cudaEventCreateWithFlags(&c->stage_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        g_create_error = std::string("sbr_create: event: ") + cudaGetErrorString(e);
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return SBR_ERR_CUDA;
    }
    c->tune.tile_w = 8;
    c->tune.blocks_per_sm = std::min(4, trace_blocks_per_sm());
    c->tune.stack_depth = 64;
    c->tune.chunk_rays_log2 = 27;
    c->tune.po_item = kPoItemRecords;
    c->tune.bvh_width = 2;
    c->tune.packet = 0;
    c->tune.silhouette = 0;
    c->tune.octant = 0;
    c->tune.raster = 1;
    *out = c;
    return SBR_OK;
}

void sbr_destroy(sbr_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    DevBuf* all[] = {&c->xyz, &c->tri, &c->nodes, &c->tris, &c->bvh_scratch, &c->bbox_dev, &c->err_dev, &c->nodes4,
                     &c->angles, &c->rayoff, &c->mask, &c->tilebase, &c->scan_scr, &c->recoff, &c->q0, &c->q1, &c->cover,
                     &c->nodes_oct, &c->tripos, &c->pool, &c->angall, &c->rayoffall, &c->recofall, &c->poolctr,
                     &c->poolwork, &c->poolgroup, &c->vis, &c->visfull, &c->hitlist, &c->rbig, &c->rbigctr, &c->ctr64, &c->ctr32, &c->stats, &c->rec, &c->hit_tri, &c->hit_t, &c->hit_nb, &c->items,
                     &c->itemoff, &c->recbeg, &c->freq, &c->kfreq, &c->partial, &c->E, &c->rcs};
    for (DevBuf* b : all) b->release();
    if (c->host_stage) cudaFreeHost(c->host_stage);
    if (c->pool_host) cudaFreeHost(c->pool_host);
    if (c->stage_ev) cudaEventDestroy(c->stage_ev);
    for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
    free_plan(c->plan);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

int sbr_load_mesh(sbr_ctx* c, const float* xyz, int64_t n_vert, const int32_t* tri, int64_t n_tri, int on_device)
{
    if (!c) return SBR_ERR_ARG;
    if (!xyz || !tri || n_vert < 3 || n_tri < 1) return fail(c, SBR_ERR_ARG, "sbr_load_mesh: empty or null mesh");
    if (n_tri >= (1ll << 27)) return fail(c, SBR_ERR_ARG, "sbr_load_mesh: at most 2^27 - 1 triangles");
    if (n_vert >= (1ll << 31)) return fail(c, SBR_ERR_ARG, "sbr_load_mesh: at most 2^31 - 1 vertices");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    c->has_mesh = c->has_bvh = c->has_trace = false;
    if (!on_device) {
        for (int64_t i = 0; i < 3 * n_tri; ++i)
            if (tri[i] < 0 || tri[i] >= n_vert) return fail(c, SBR_ERR_ARG, "sbr_load_mesh: index %lld out of range", (long long)i);
        for (int64_t i = 0; i < 3 * n_vert; ++i)
            if (!std::isfinite(xyz[i]))
                return fail(c, SBR_ERR_ARG, "sbr_load_mesh: vertex coordinate %lld is not finite", (long long)i);
    }
    CK(c->xyz.ensure(sizeof(float) * 3 * (size_t)n_vert), "alloc xyz");
    CK(c->tri.ensure(sizeof(int32_t) * 3 * (size_t)n_tri), "alloc tri");
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(c->xyz.p, xyz, sizeof(float) * 3 * (size_t)n_vert, kind, c->stream), "copy xyz");
    CK(cudaMemcpyAsync(c->tri.p, tri, sizeof(int32_t) * 3 * (size_t)n_tri, kind, c->stream), "copy tri");
    c->n_vert = n_vert;
    c->n_tri = n_tri;
    // exact scene box and index check run as part of the BVH build; build the
    // box now so sbr_get_bbox / sbr_ray_grid_for work right after loading
    c->has_mesh = true;
    return sbr_build_bvh(c, nullptr);
}

int sbr_get_bbox(sbr_ctx* c, float* bbox6)
{
    if (!c || !bbox6) return SBR_ERR_ARG;
    if (!c->has_mesh) return fail(c, SBR_ERR_STATE, "sbr_get_bbox: no mesh loaded");
    memcpy(bbox6, c->bbox, sizeof(c->bbox));
    return SBR_OK;
}

int sbr_build_bvh(sbr_ctx* c, const sbr_bvh_opts* opt)
{
    if (!c) return SBR_ERR_ARG;
    if (!c->has_mesh) return fail(c, SBR_ERR_STATE, "sbr_build_bvh: no mesh loaded");
    int leaf_max = opt ? opt->leaf_max : 4;
    float ct = opt ? opt->cost_traverse : 1.f, ci = opt ? opt->cost_intersect : 1.f;
    if (leaf_max < 1 || leaf_max > kLeafMax) return fail(c, SBR_ERR_ARG, "sbr_build_bvh: leaf_max must be 1..16");
    if (!(ct >= 0.f) || !(ci > 0.f)) return fail(c, SBR_ERR_ARG, "sbr_build_bvh: costs must be C_T >= 0, C_I > 0");
    const int builder = opt ? opt->builder : SBR_BVH_PLOC, radius = opt ? opt->ploc_radius : 0;
    if (builder != SBR_BVH_LBVH && builder != SBR_BVH_PLOC) return fail(c, SBR_ERR_ARG, "sbr_build_bvh: unknown builder");
    if (radius < 0 || radius > 64) return fail(c, SBR_ERR_ARG, "sbr_build_bvh: ploc_radius must be 0..64");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    ++c->mesh_gen;  // captured batch graphs hold the node and triangle pointers
    const long long n = c->n_tri;
    const long long n_nodes = n > 1 ? n - 1 : 1;
    c->n_nodes = n_nodes;
    CK(c->nodes.ensure(sizeof(float4) * 4 * (size_t)n_nodes), "alloc nodes");
    // records (3 float4), normals (1) and exact v1, v2 (2) per triangle
    CK(c->tris.ensure(sizeof(float4) * 6 * (size_t)n), "alloc tris");
    CK(c->tripos.ensure(sizeof(int) * (size_t)n), "alloc triangle positions");
    size_t sb = bvh_scratch_bytes(n);
    CK(c->bvh_scratch.ensure(sb), "alloc bvh scratch");
    CK(c->bbox_dev.ensure(sizeof(float) * 8), "alloc bbox");
    CK(c->err_dev.ensure(sizeof(int) * 4), "alloc err");
    BvhBuild b;
    b.xyz = c->xyz.as<float>();
    b.tri = c->tri.as<int>();
    b.n_vert = c->n_vert;
    b.n_tri = n;
    b.leaf_max = leaf_max;
    b.c_t = ct;
    b.c_i = ci;
    b.builder = builder == SBR_BVH_PLOC ? 1 : 0;
    b.radius = radius;
    b.nodes = c->nodes.as<float4>();
    b.tris = c->tris.as<float4>();
    b.tri_nrm = c->tris.as<float4>() + 3 * (size_t)n;
    b.tri_v12 = c->tris.as<float4>() + 4 * (size_t)n;
    b.tri_pos = c->tripos.as<int>();
    b.bbox_out = c->bbox_dev.as<float>();
    b.err_flag = c->err_dev.as<int>();
    b.n_nodes_out = c->err_dev.as<int>() + 2;
    b.scratch = c->bvh_scratch.p;
    b.scratch_bytes = c->bvh_scratch.cap;
    CK(bvh_build(b, c->stream), "bvh build");
    float hb[8];
    int herr[3] = {0, 0, 0};
    CK(cudaMemcpyAsync(hb, c->bbox_dev.p, sizeof(float) * 6, cudaMemcpyDeviceToHost, c->stream), "copy bbox");
    CK(cudaMemcpyAsync(herr, c->err_dev.p, sizeof(int) * 3, cudaMemcpyDeviceToHost, c->stream), "copy err");
    CK(cudaStreamSynchronize(c->stream), "bvh build sync");
    if (herr[0]) {
        c->has_mesh = false;
        if (herr[0] & 4) return fail(c, SBR_ERR_CUDA, "sbr_build_bvh: the clustering did not converge");
        return fail(c, SBR_ERR_ARG, (herr[0] & 1) ? "sbr_build_bvh: triangle index out of range"
                                                  : "sbr_build_bvh: a vertex coordinate is not finite");
    }
    // the nodes reachable from the root, renumbered 0.. in depth-first order
    if (herr[2] < 1 || herr[2] > n_nodes) {
        c->has_mesh = false;
        return fail(c, SBR_ERR_CUDA, "sbr_build_bvh: malformed hierarchy (%d reachable nodes of %lld)", herr[2],
                    n_nodes);
    }
    c->n_nodes = herr[2];
    memcpy(c->bbox, hb, sizeof(c->bbox));
    // 4-wide tree over the same boxes; its work queues reuse the (now free) build scratch
    CK(c->nodes4.ensure(sizeof(float4) * kNode4Float4 * (size_t)c->n_nodes), "alloc 4-wide nodes");
    {
        char* scr = (char*)c->bvh_scratch.p;
        const size_t qb = ((sizeof(int2) * (size_t)c->n_nodes + 255) / 256) * 256;
        if (2 * qb + 256 > c->bvh_scratch.cap) return fail(c, SBR_ERR_ARG, "sbr_build_bvh: scratch too small");
        CK(bvh4_collapse(c->nodes.as<float4>(), c->n_nodes, c->nodes4.as<float4>(), (int2*)scr, (int2*)(scr + qb),
                         (int*)(scr + 2 * qb), &c->n_nodes4, c->stream),
           "4-wide collapse");
    }
    c->has_bvh = true;
    c->has_trace = false;
    return SBR_OK;
}

int sbr_get_bvh_info(sbr_ctx* c, sbr_bvh_info* out)
{
    if (!c || !out) return SBR_ERR_ARG;
    if (!c->has_bvh) return fail(c, SBR_ERR_STATE, "sbr_get_bvh_info: no tree built");
    out->n_tri = c->n_tri;
    out->n_nodes = c->n_nodes;
    out->n_nodes4 = c->n_nodes4;
    return SBR_OK;
}

int sbr_ray_grid_for(sbr_ctx* c, double az_deg, double el_deg, double ds, double eta, const sbr_trace_opts* opt,
                     sbr_ray_grid* out)
{
    if (!c || !out) return SBR_ERR_ARG;
    if (!c->has_mesh) return fail(c, SBR_ERR_STATE, "sbr_ray_grid_for: no mesh loaded");
    if (!(ds > 0.0) || !(eta >= 0.0)) return fail(c, SBR_ERR_ARG, "sbr_ray_grid_for: spacing must be > 0, eta >= 0");
    make_grid(c->bbox, az_deg, el_deg, ds, eta, opt, out);
    return SBR_OK;
}

int sbr_ray_grid_box(const float* bbox6, double az_deg, double el_deg, double ds, double eta, const sbr_trace_opts* opt,
                 sbr_ray_grid* out)
{
    if (!bbox6 || !out) return SBR_ERR_ARG;
    if (!(ds > 0.0) || !(eta >= 0.0)) return SBR_ERR_ARG;
    make_grid(bbox6, az_deg, el_deg, ds, eta, opt, out);
    return SBR_OK;
}

}  // extern "C"

namespace {

// per-call state of a trace (sbr_trace or sbr_run_batch)
struct TraceRun {
    int flags = 0, max_bounces = 1;
    bool escape = false, hits = false, count = false, timed = false;
    long long chunk_cap = 1ll << 27;
    int stop_after = -1;  // >= 0: a chunk runs its bounce passes up to this one only (the rest are pooled)
    RayState* pool = nullptr;  // with stop_after: the chunk's last pass appends the rays that go on here
    unsigned* pool_count = nullptr;
    unsigned pool_cap = 0;
    int n_blocks = 0;
    int64_t n_launch = 0, n_pass = 0;
    size_t n_ev = 0;
    std::vector<char> ev_primary;  // per timed pass: 1 for a primary pass
};

// Lay out the aspects c->ang[0..n) (grids filled) in processing order, cut them
// into chunks of at most chunk_cap rays and size the per-chunk buffers.
int plan_chunks(sbr_ctx* c, TraceRun& R, std::vector<int64_t>& cut, long long* total_out, long long* launched_out)
{
    const int64_t n = (int64_t)c->ang.size();
    long long total = 0, launched = 0;
    for (int64_t a = 0; a < n; ++a) {
        AngleHost& h = c->ang[(size_t)a];
        if (h.grid.nu > (1ll << 30) || h.grid.nv > (1ll << 30) || tiled_rays(h.grid, h.tw) > R.chunk_cap)
            return fail(c, SBR_ERR_ARG, "ray grid of aspect %lld too large (%lld x %lld) for a chunk of %lld rays",
                        (long long)a, (long long)h.grid.nu, (long long)h.grid.nv, R.chunk_cap);
        h.ray_begin = total;
        h.rec_begin = h.rec_count = 0;
        total += tiled_rays(h.grid, h.tw);
        launched += h.grid.nu * h.grid.nv;
    }
    cut.assign(1, 0);
    long long acc = 0;
    for (int64_t a = 0; a < n; ++a) {
        const long long r = tiled_rays(c->ang[(size_t)a].grid, c->ang[(size_t)a].tw);
        if (acc > 0 && acc + r > R.chunk_cap) {
            cut.push_back(a);
            acc = 0;
        }
        acc += r;
    }
    cut.push_back(n);
    long long max_chunk = 0;
    int max_angles = 0;
    for (size_t k = 0; k + 1 < cut.size(); ++k) {
        const AngleHost& last = c->ang[(size_t)cut[k + 1] - 1];
        max_chunk = std::max(max_chunk, last.ray_begin + tiled_rays(last.grid, last.tw) - c->ang[(size_t)cut[k]].ray_begin);
        max_angles = std::max(max_angles, (int)(cut[k + 1] - cut[k]));
    }
    const long long max_tiles = max_chunk / 32;
    // hit masks and their prefix for the whole trace (a chunk uses its own range): the pooled late passes
    // find the record slot of a ray of any chunk
    const long long all_tiles = total / 32;
    CK(c->angles.ensure(sizeof(AngleDev) * (size_t)max_angles), "alloc angles");
    CK(c->rayoff.ensure(sizeof(long long) * (size_t)(max_angles + 1)), "alloc ray offsets");
    CK(c->recoff.ensure(sizeof(unsigned) * (size_t)(max_angles + 1)), "alloc record offsets");
    CK(c->mask.ensure(sizeof(unsigned) * (size_t)all_tiles), "alloc mask");
    if (c->tune.silhouette) CK(c->cover.ensure(sizeof(unsigned) * (size_t)(max_tiles + max_angles)), "alloc cover");
    if (c->tune.raster) {
        CK(c->vis.ensure(sizeof(unsigned long long) * (size_t)max_chunk), "alloc raster keys");
        CK(c->visfull.ensure(sizeof(unsigned) * (size_t)(max_angles + 1)), "alloc raster flags");
        CK(c->hitlist.ensure(sizeof(uint2) * (size_t)max_chunk), "alloc raster hit list");
        c->rbig_cap = raster_big_cap(max_chunk);
        CK(c->rbig.ensure(sizeof(int4) * (size_t)c->rbig_cap), "alloc raster triangle list");
        CK(c->rbigctr.ensure(sizeof(unsigned) * 2), "alloc raster triangle counters");
    }
    CK(c->tilebase.ensure(sizeof(unsigned) * (size_t)all_tiles), "alloc tile base");
    CK(c->scan_scr.ensure(scan_scratch_bytes(max_tiles)), "alloc scan scratch");
    CK(c->q0.ensure(sizeof(RayState) * (size_t)max_chunk), "alloc ray queue");
    CK(c->q1.ensure(sizeof(RayState) * (size_t)max_chunk), "alloc ray queue");
    CK(c->ctr64.ensure(sizeof(unsigned long long) * 2 * (kMaxBounces + 2)), "alloc counters");
    CK(c->ctr32.ensure(sizeof(unsigned) * 2 * (kMaxBounces + 2) + 64), "alloc counters");
    CK(c->stats.ensure(sizeof(unsigned long long) * kStatCount), "alloc stats");
    CK(cudaMemsetAsync(c->stats.p, 0, sizeof(unsigned long long) * kStatCount, c->stream), "memset stats");
    if (R.hits) {
        const size_t B = (size_t)R.max_bounces;
        CK(c->hit_tri.ensure(sizeof(int) * (size_t)total * B), "alloc hit ids");
        CK(c->hit_t.ensure(sizeof(float) * (size_t)total * B), "alloc hit t");
        CK(c->hit_nb.ensure(sizeof(int) * (size_t)total), "alloc hit counts");
        CK(cudaMemsetAsync(c->hit_tri.p, 0xFF, sizeof(int) * (size_t)total * B, c->stream), "memset");
        CK(cudaMemsetAsync(c->hit_t.p, 0, sizeof(float) * (size_t)total * B, c->stream), "memset");
        CK(cudaMemsetAsync(c->hit_nb.p, 0, sizeof(int) * (size_t)total, c->stream), "memset");
    }
    R.n_blocks = c->n_sms * c->tune.blocks_per_sm;
    *total_out = total;
    *launched_out = launched;
    return SBR_OK;
}

cudaEvent_t pool_event(sbr_ctx* c, size_t i)
{
    while (c->evpool.size() <= i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->evpool.push_back(e);
    }
    return c->evpool[i];
}

// the octant copies of the current binary nodes (built once per tree)
cudaError_t ensure_octant_nodes(sbr_ctx* c, cudaStream_t st)
{
    if (c->oct_gen == c->mesh_gen) return cudaSuccess;
    cudaError_t e = c->nodes_oct.ensure(sizeof(float4) * 4 * 8 * (size_t)c->n_nodes);
    if (e == cudaSuccess) e = build_octant_nodes(c->nodes.as<float4>(), c->n_nodes, c->nodes_oct.as<float4>(), st);
    if (e == cudaSuccess) c->oct_gen = c->mesh_gen;
    return e;
}

// Enqueue the trace of the aspects [a0, a1) (one chunk): primary pass, popcount
// scan of the hit masks, bounce passes, and the copy of the per-aspect record
// offsets to *hro_out (pinned). Nothing waits for the GPU: the record buffer is
// sized for every ray of the chunk being valid. Records go to c->rec from index
// rec_base on; earlier records are kept. chunk_records reads *hro_out once the
// stream has passed it.
// a transport pass; the primary pass includes the rasterisation of its hits
cudaError_t run_pass(sbr_ctx* c, TraceRun& R, const TraceArgs& t)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (R.timed) {
        e0 = pool_event(c, R.n_ev);
        e1 = pool_event(c, R.n_ev + 1);
        if (!e0 || !e1) return cudaErrorMemoryAllocation;
        R.n_ev += 2;
        R.ev_primary.push_back(t.bounce == 0 ? 1 : 0);
        cudaEventRecord(e0, c->stream);
    }
    cudaError_t e = cudaSuccess;
    if (t.vis && t.bounce == 0) {
        e = launch_raster(t, (int)c->n_tri, c->vis.as<unsigned long long>(), c->visfull.as<unsigned>(), R.count,
                          c->n_sms * 16, c->scan_scr.p, c->stream);
        R.n_launch += 6;  // rasterisation, masks, 3-kernel scan, primary pass of the rasterised rays
    }
    if (e == cudaSuccess) e = launch_trace(t, R.n_blocks, R.count, c->tune.stack_depth, c->stream);
    if (R.timed) cudaEventRecord(e1, c->stream);
    ++R.n_launch;
    ++R.n_pass;
    return e;
}

int trace_chunk(sbr_ctx* c, TraceRun& R, int64_t a0, int64_t a1, long long rec_base, unsigned** hro_out)
{
    const int na = (int)(a1 - a0);
    const long long base = c->ang[(size_t)a0].ray_begin;
    const long long chunk_rays = c->ang[(size_t)a1 - 1].ray_begin +
                                 tiled_rays(c->ang[(size_t)a1 - 1].grid, c->ang[(size_t)a1 - 1].tw) - base;
    unsigned* q_count = c->ctr32.as<unsigned>();
    unsigned* total_dev = q_count + 2 * (kMaxBounces + 2);
    // the chunk's range of the trace-wide hit masks and their prefix (base is a multiple of 32)
    unsigned* mask = c->mask.as<unsigned>() + base / 32;
    unsigned* tilebase = c->tilebase.as<unsigned>() + base / 32;
    auto pass = [&](const TraceArgs& t) -> cudaError_t { return run_pass(c, R, t); };
    // stage angle table and ray offsets
    const size_t bytes_a = sizeof(AngleDev) * (size_t)na, bytes_o = sizeof(long long) * (size_t)(na + 1);
    char* hs = (char*)stage(c, bytes_a + bytes_o + sizeof(unsigned) * (size_t)(na + 1));
    if (!hs) return fail(c, SBR_ERR_OOM, "pinned staging allocation failed");
    // grow the record buffer to the worst case, keeping the records below rec_base
    const size_t need = sizeof(Record) * (size_t)(rec_base + chunk_rays);
    if (need > c->rec.cap) {
        DevBuf nb;
        CK(nb.ensure(need + need / 4), "alloc records");
        cudaError_t e = cudaSuccess;
        if (rec_base > 0)
            e = cudaMemcpyAsync(nb.p, c->rec.p, sizeof(Record) * (size_t)rec_base, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            nb.release();
            return cuda_fail(c, e, "copy records");
        }
        c->rec.release();
        c->rec = nb;
    }
    AngleDev* ha = (AngleDev*)hs;
    long long* ho = (long long*)(hs + bytes_a);
    for (int i = 0; i < na; ++i) {
        const AngleHost& h = c->ang[(size_t)(a0 + i)];
        ho[i] = h.ray_begin - base;
        double rx[2] = {h.rx_az, h.rx_el};
        ha[i] = to_dev(h.grid, ho[i], h.tw, h.bistatic ? rx : nullptr);
    }
    ho[na] = chunk_rays;
    CK(cudaMemcpyAsync(c->angles.p, ha, bytes_a, cudaMemcpyHostToDevice, c->stream), "copy angles");
    CK(cudaMemcpyAsync(c->rayoff.p, ho, bytes_o, cudaMemcpyHostToDevice, c->stream), "copy ray offsets");
    CK(cudaMemsetAsync(c->ctr64.p, 0, c->ctr64.cap, c->stream), "memset counters");
    CK(cudaMemsetAsync(c->ctr32.p, 0, c->ctr32.cap, c->stream), "memset counters");
    TraceArgs ta;
    memset(&ta, 0, sizeof(ta));
    ta.wide = c->tune.bvh_width == 4;
    ta.packet = c->tune.packet;
    ta.octant = c->tune.octant;
    ta.n_nodes = c->n_nodes;
    for (int i = 0; i < na; ++i) ta.bistatic |= c->ang[(size_t)(a0 + i)].bistatic ? 1 : 0;
    if (ta.octant) CK(ensure_octant_nodes(c, c->stream), "octant nodes");
    ta.nodes = ta.wide ? c->nodes4.as<float4>() : (ta.octant ? c->nodes_oct.as<float4>() : c->nodes.as<float4>());
    ta.tris = c->tris.as<float4>();
    ta.tri_nrm = ta.tris + 3 * (size_t)c->n_tri;
    ta.tri_v12 = ta.tris + 4 * (size_t)c->n_tri;
    ta.angles = c->angles.as<AngleDev>();
    ta.ray_off = c->rayoff.as<long long>();
    ta.n_angles = na;
    ta.max_bounces = R.max_bounces;
    ta.flags = R.flags;
    ta.visit_limit = (int)std::min<long long>(2 * c->n_tri + 64, 1ll << 30);
    ta.total_rays = chunk_rays;
    ta.mask = mask;
    ta.tile_base = tilebase;
    ta.stats = c->stats.as<unsigned long long>();
    if (R.hits) {
        ta.hit_tri = c->hit_tri.as<int>() + (size_t)base * R.max_bounces;
        ta.hit_t = c->hit_t.as<float>() + (size_t)base * R.max_bounces;
        ta.hit_nb = c->hit_nb.as<int>() + base;
    }
    RayState* qs[2] = {c->q0.as<RayState>(), c->q1.as<RayState>()};
    if (c->tune.raster) {  // primary hits by rasterisation (the silhouette mask is then not needed)
        ta.vis = c->vis.as<unsigned long long>();
        ta.vis_full = c->visfull.as<unsigned>();
        ta.big = c->rbig.as<int4>();
        ta.big_ctr = c->rbigctr.as<unsigned>();
        ta.big_cap = (unsigned)c->rbig_cap;
        ta.tri_pos = c->tripos.as<int>();
        ta.list_count = total_dev + 4;
        // a bounce pass follows: list the hits and let it rebuild their states (not for B = 1, whose
        // records are written from the stored states, nor for bistatic chunks; binary traversals only,
        // where the rebuilding fits the bounce kernel's registers)
        if (!ta.bistatic && !ta.wide && !ta.packet && (R.max_bounces >= 2 || R.escape))
            ta.hit_list = c->hitlist.as<uint2>();
    } else if (c->tune.silhouette) {
        CK(cudaMemsetAsync(c->cover.p, 0, sizeof(unsigned) * (size_t)(chunk_rays / 32 + na), c->stream), "memset cover");
        CK(launch_silhouette(ta, (int)c->n_tri, c->cover.as<unsigned>(), c->stream), "silhouette");
        ++R.n_launch;
        ta.cover = c->cover.as<unsigned>();
    }
    ta.bounce = 0;  // pass 0: primary rays -> queue 0
    ta.work = c->ctr64.as<unsigned long long>();
    ta.q_out = qs[0];
    ta.q_out_count = q_count + 1;
    CK(pass(ta), "trace primary");
    CK(scan_popc(ta.mask, tilebase, chunk_rays / 32, total_dev, c->scan_scr.p, c->stream), "scan");
    R.n_launch += 3;
    CK(launch_angle_offsets(ta.ray_off, tilebase, total_dev, na, c->recoff.as<unsigned>(), c->stream),
       "angle offsets");
    ++R.n_launch;
    unsigned* hro = (unsigned*)(hs + bytes_a + bytes_o);
    CK(cudaMemcpyAsync(hro, c->recoff.p, sizeof(unsigned) * (size_t)(na + 1), cudaMemcpyDeviceToHost, c->stream),
       "copy record offsets");
    CK(cudaEventRecord(c->stage_ev, c->stream), "record staging event");
    *hro_out = hro;
    ta.rec = c->rec.as<Record>() + rec_base;
    if (R.max_bounces == 1 && !R.escape) {
        ta.q_in = qs[0];
        ta.q_in_count = q_count + 1;
        CK(launch_emit_all(ta, R.n_blocks, c->stream), "emit");
        ++R.n_launch;
    } else {
        int last_pass = R.escape ? R.max_bounces : R.max_bounces - 1;
        if (R.stop_after >= 0) last_pass = std::min(last_pass, R.stop_after);
        for (int b = 1; b <= last_pass; ++b) {
            ta.bounce = b;
            ta.work = c->ctr64.as<unsigned long long>() + b;
            ta.q_in = qs[(b - 1) & 1];
            ta.q_in_count = q_count + b;
            ta.q_out = qs[b & 1];
            ta.q_out_count = q_count + b + 1;
            if (R.pool && b == last_pass) {  // the rays that go on join the ray pool (those it cannot take: q_out)
                ta.pool = R.pool;
                ta.pool_count = R.pool_count;
                ta.pool_cap = R.pool_cap;
                ta.angle_shift = (int)a0;
            }
            CK(pass(ta), "trace bounce");
            ta.hit_list = nullptr;  // only bounce pass 1 reads the list
        }
    }
    return SBR_OK;
}

// the record range of each aspect of the chunk [a0, a1) from the offsets that
// trace_chunk copied to hro (the stream must have passed that copy); returns the
// chunk's record count
long long chunk_records(sbr_ctx* c, int64_t a0, int64_t a1, long long rec_base, const unsigned* hro)
{
    const int na = (int)(a1 - a0);
    for (int i = 0; i < na; ++i) {
        AngleHost& h = c->ang[(size_t)(a0 + i)];
        h.rec_begin = rec_base + hro[i];
        h.rec_count = (long long)hro[i + 1] - hro[i];
    }
    return hro[na];
}

// wait for the stream and read the device counters
int read_counters(sbr_ctx* c, unsigned long long* hs_stats)
{
    CK(cudaMemcpyAsync(hs_stats, c->stats.p, sizeof(unsigned long long) * kStatCount, cudaMemcpyDeviceToHost,
                       c->stream),
       "copy stats");
    CK(cudaStreamSynchronize(c->stream), "trace end sync");
    return SBR_OK;
}

// fill stats from the counters read by read_counters; SBR_ERR_STACK_OVERFLOW if any traversal overflowed
int finish_stats(sbr_ctx* c, const TraceRun& R, const unsigned long long* hs_stats, int64_t n_angles,
                 long long launched, long long valid, sbr_trace_stats* stats)
{
    if (stats) {
        stats->n_angles = n_angles;
        stats->rays_launched = launched;
        stats->ray_bounces = (int64_t)hs_stats[kStatQueries];
        stats->valid_rays = valid;
        stats->node_visits = (int64_t)hs_stats[kStatNodes];
        stats->tri_tests = (int64_t)hs_stats[kStatTris];
        stats->stack_overflows = (int64_t)hs_stats[kStatOverflow];
        stats->kernel_launches = R.n_launch;
        stats->pass_launches = R.n_pass;
        stats->raster_tests = (int64_t)hs_stats[kStatRaster];
        stats->bounce_hits = (int64_t)hs_stats[kStatHits];
        stats->listed_hits = (int64_t)hs_stats[kStatListed];
        stats->open_tests = (int64_t)hs_stats[kStatOpen];
        stats->fp64_tests = (int64_t)hs_stats[kStatFp64];
        stats->warp_node_visits = (int64_t)hs_stats[kStatWarpNodes];
        stats->pass_ms = 0.0;
        stats->primary_ms = 0.0;
        for (size_t i = 0; R.timed && i + 1 < R.n_ev; i += 2) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, c->evpool[i], c->evpool[i + 1]) == cudaSuccess) {
                stats->pass_ms += ms;
                if (R.ev_primary[i / 2]) stats->primary_ms += ms;
            }
        }
    }
    if (hs_stats[kStatOverflow])
        return fail(c, SBR_ERR_STACK_OVERFLOW, "%llu traversals exceeded the stack depth",
                    (unsigned long long)hs_stats[kStatOverflow]);
    return SBR_OK;
}

int check_po_mode(sbr_ctx* c, int pol_mask, int po_mode, PoArgs& pa)
{
    if (pol_mask <= 0 || pol_mask > 15) return fail(c, SBR_ERR_ARG, "pol_mask must select HH/VV/HV/VH");
    const int form = po_mode & 15, prec = po_mode & ~15;
    if (form != SBR_PO_VECTOR && form != SBR_PO_PAPER_SCALAR) return fail(c, SBR_ERR_ARG, "unknown PO form");
    if (prec != SBR_PHASE_COMPENSATED && prec != SBR_PHASE_FP32 && prec != SBR_PHASE_FP64)
        return fail(c, SBR_ERR_ARG, "unknown phase precision");
    memset(&pa, 0, sizeof(pa));
    for (int q = 0; q < 4; ++q)
        if (pol_mask & (1 << q)) pa.pol_sel[pa.n_pol++] = q;
    pa.scalar = form == SBR_PO_PAPER_SCALAR;
    pa.phase_mode = prec == SBR_PHASE_COMPENSATED ? 0 : (prec == SBR_PHASE_FP32 ? 1 : 2);
    return SBR_OK;
}

// upload the frequency table: (kappa_hi, kappa_lo, k) per frequency, kappa = f / c0
int upload_freqs(sbr_ctx* c, const double* freq_hz, int64_t n_freq)
{
    for (int64_t f = 0; f < n_freq; ++f)
        if (!(freq_hz[f] > 0.0)) return fail(c, SBR_ERR_ARG, "frequencies must be > 0");
    const size_t b_freq = sizeof(float4) * (size_t)n_freq, b_kf = sizeof(double) * (size_t)n_freq;
    CK(c->freq.ensure(b_freq), "alloc freq");
    CK(c->kfreq.ensure(b_kf), "alloc freq");
    char* hs = (char*)stage(c, b_freq + b_kf + 64);
    if (!hs) return fail(c, SBR_ERR_OOM, "pinned staging allocation failed");
    float4* hf = (float4*)hs;
    double* hk = (double*)(hs + b_freq);
    for (int64_t f = 0; f < n_freq; ++f) {
        const double kappa = freq_hz[f] / kC0;  // cycles per metre
        const float kh = (float)kappa;
        const double k = 2.0 * kPi * freq_hz[f] / kC0;
        hf[f] = make_float4(kh, (float)(kappa - (double)kh), (float)k, 0.f);
        hk[f] = k;
    }
    CK(cudaMemcpyAsync(c->freq.p, hf, b_freq, cudaMemcpyHostToDevice, c->stream), "copy freq");
    CK(cudaMemcpyAsync(c->kfreq.p, hk, b_kf, cudaMemcpyHostToDevice, c->stream), "copy freq");
    CK(cudaEventRecord(c->stage_ev, c->stream), "record staging event");
    return SBR_OK;
}

// PO sum of the aspects [a0, a1) of c->ang over their records; aspect a uses
// frequencies [f0[a], f0[a] + nf[a]) of the uploaded table and writes rows
// out_row[a] .. of the device outputs dE / dR.
int po_run(sbr_ctx* c, PoArgs pa, int64_t a0, int64_t a1, const std::vector<int>& f0, const std::vector<int>& nf,
           const std::vector<long long>& out_row, double* dE, double* dR, int64_t* n_launch)
{
    // per-aspect tables on the host (item ranges, partial offsets, record offsets); a kernel expands them
    // into the work list, so the host never touches the items
    const int na = (int)(a1 - a0);
    const int per = c->tune.po_item;
    const size_t b_ang = sizeof(PoAngle) * (size_t)na, b_off = sizeof(long long) * (size_t)(na + 1);
    char* hs = (char*)stage(c, b_ang + b_off);
    if (!hs) return fail(c, SBR_ERR_OOM, "pinned staging allocation failed");
    PoAngle* pang = (PoAngle*)hs;
    long long* off = (long long*)(hs + b_ang);
    long long part = 0, n_items = 0;
    for (int i = 0; i < na; ++i) {
        const AngleHost& h = c->ang[(size_t)(a0 + i)];
        if (i > 0 && h.rec_begin != off[i])
            return fail(c, SBR_ERR_STATE, "records of consecutive aspects are not contiguous");
        off[i] = h.rec_begin;
        off[i + 1] = h.rec_begin + h.rec_count;
        PoAngle& A = pang[(size_t)i];
        const long long ni = (h.rec_count + per - 1) / per;
        A.item_begin = (int)n_items;
        A.item_end = (int)(n_items + ni);
        A.f0 = f0[(size_t)(a0 + i)];
        A.nf = nf[(size_t)(a0 + i)];
        A.out_row = out_row[(size_t)(a0 + i)];
        A.part = part;
        n_items += ni;
        part += ni * A.nf * 2 * pa.n_pol;
    }
    if (n_items >= (1ll << 31)) return fail(c, SBR_ERR_ARG, "too many PO work items");
    CK(c->items.ensure(std::max(sizeof(PoItem) * (size_t)n_items, (size_t)32)), "alloc items");
    CK(c->itemoff.ensure(b_ang), "alloc aspect table");
    CK(c->recbeg.ensure(b_off), "alloc record offsets");
    CK(c->partial.ensure(sizeof(double) * (size_t)std::max(part, 1ll)), "alloc partials");
    CK(cudaMemcpyAsync(c->itemoff.p, pang, b_ang, cudaMemcpyHostToDevice, c->stream), "copy aspect table");
    CK(cudaMemcpyAsync(c->recbeg.p, off, b_off, cudaMemcpyHostToDevice, c->stream), "copy record offsets");
    CK(cudaEventRecord(c->stage_ev, c->stream), "record staging event");
    if (n_items > 0)
        CK(launch_po_items_fill(c->recbeg.as<long long>(), c->itemoff.as<PoAngle>(), na, pa.n_pol, per,
                                c->items.as<PoItem>(), c->stream),
           "po work list");
    pa.rec = c->rec.as<Record>();
    pa.items = c->items.as<PoItem>();
    pa.n_items = (int)n_items;
    pa.freq = c->freq.as<float4>();
    pa.kfreq = c->kfreq.as<double>();
    pa.partial = c->partial.as<double>();
    pa.item_records = c->tune.po_item;
    pa.err = c->err_dev.as<int>() + 3;  // bounded waits of the staged single-frequency sum (callers clear it)
    CK(launch_po(pa, c->stream), "po reduce");
    CK(launch_po_final(pa.partial, pa.items, c->itemoff.as<PoAngle>(), na, pa.kfreq, pa.n_pol, dE, dR, c->stream),
       "po final");
    if (n_launch) *n_launch += (n_items > 0 ? 2 : 0) + 1;
    return SBR_OK;
}

// ---------------------------------------------------------------- asynchronous batches
// A plan holds one submitted batch: its ray grids cut into chunks, device
// tables uploaded once, buffers sized for the worst case (every ray valid) and
// the captured CUDA graph of the whole batch.
struct BatchPlan {
    // identity of the submission
    std::vector<sbr_request> req;
    std::vector<double> freq;
    double eta = 0.0;
    int max_bounces = 0, pol_mask = 0, po_mode = 0, flags = 0;
    sbr_tuning tune;
    sbr_trace_opts opt;
    double* E = nullptr;
    double* R = nullptr;
    long long mesh_gen = -1;
    // chunks of aspects [cut[k], cut[k + 1])
    std::vector<int64_t> cut;
    std::vector<long long> chunk_rays, items_bound;
    long long launched = 0;
    int64_t n_launch = 0, n_pass = 0;
    bool count = false;
    unsigned big_cap = 0;  // entries of rbig
    PoArgs pa;
    // device buffers
    DevBuf angles, rayoff, pang, recoff, mask, tilebase, scan_scr, q0, q1, ctr64, ctr32, stats, rec, items, nitems,
        valid, freq_t, kfreq, partial, cover, vis, visfull, hitlist, rbig, rbigctr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

void free_plan(BatchPlan* p)
{
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->cap) cudaStreamDestroy(p->cap);
    DevBuf* all[] = {&p->angles, &p->rayoff, &p->pang,   &p->recoff, &p->mask,   &p->tilebase, &p->scan_scr,
                     &p->q0,     &p->q1,     &p->ctr64,  &p->ctr32,  &p->stats,  &p->rec,      &p->items,
                     &p->nitems, &p->valid,  &p->freq_t, &p->kfreq,  &p->partial, &p->cover,
                     &p->vis,    &p->visfull, &p->hitlist, &p->rbig, &p->rbigctr};
    for (DevBuf* b : all) b->release();
    delete p;
}

bool same_submission(const BatchPlan& P, const sbr_ctx* c, const sbr_request* req, int64_t n_req, const double* freq,
                     int64_t n_freq, double eta, int max_bounces, int pol_mask, int po_mode, const sbr_trace_opts& o,
                     double* E, double* R)
{
    return P.mesh_gen == c->mesh_gen && memcmp(&P.tune, &c->tune, sizeof(sbr_tuning)) == 0 &&
           (int64_t)P.req.size() == n_req &&
           (int64_t)P.freq.size() == n_freq && P.eta == eta && P.max_bounces == max_bounces &&
           P.pol_mask == pol_mask && P.po_mode == po_mode && P.E == E && P.R == R &&
           memcmp(&P.opt, &o, sizeof(o)) == 0 && memcmp(P.req.data(), req, sizeof(sbr_request) * (size_t)n_req) == 0 &&
           memcmp(P.freq.data(), freq, sizeof(double) * (size_t)n_freq) == 0;
}

// Enqueue the whole batch on stream st: per chunk the transport passes, the
// record scan, the device-built PO work list, the PO sums and the final sums.
cudaError_t enqueue_plan(const sbr_ctx* c, BatchPlan& P, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(P.stats.p, 0, sizeof(unsigned long long) * kStatCount, st);
    unsigned* q_count = P.ctr32.as<unsigned>();
    unsigned* total_dev = q_count + 2 * (kMaxBounces + 2);
    RayState* qs[2] = {P.q0.as<RayState>(), P.q1.as<RayState>()};
    const int n_blocks = c->n_sms * P.tune.blocks_per_sm;
    const bool escape = P.flags & SBR_TRACE_REQUIRE_ESCAPE;
    for (size_t k = 0; e == cudaSuccess && k + 1 < P.cut.size(); ++k) {
        const int64_t a0 = P.cut[k];
        const int na = (int)(P.cut[k + 1] - a0);
        const long long rays = P.chunk_rays[k];
        e = cudaMemsetAsync(P.ctr64.p, 0, P.ctr64.cap, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(P.ctr32.p, 0, P.ctr32.cap, st);
        if (e != cudaSuccess) break;
        TraceArgs ta;
        memset(&ta, 0, sizeof(ta));
        ta.wide = P.tune.bvh_width == 4;
        ta.packet = P.tune.packet;
        ta.octant = P.tune.octant;
        ta.n_nodes = c->n_nodes;
        ta.nodes = ta.wide ? c->nodes4.as<float4>() : (ta.octant ? c->nodes_oct.as<float4>() : c->nodes.as<float4>());
        ta.tris = c->tris.as<float4>();
        ta.tri_nrm = ta.tris + 3 * (size_t)c->n_tri;
        ta.tri_v12 = ta.tris + 4 * (size_t)c->n_tri;
        ta.angles = P.angles.as<AngleDev>() + a0;
        ta.ray_off = P.rayoff.as<long long>() + a0 + (int64_t)k;  // chunk k's table has na + 1 entries
        ta.n_angles = na;
        ta.max_bounces = P.max_bounces;
        ta.flags = P.flags;
        ta.visit_limit = (int)std::min<long long>(2 * c->n_tri + 64, 1ll << 30);
        ta.total_rays = rays;
        ta.mask = P.mask.as<unsigned>();
        ta.tile_base = P.tilebase.as<unsigned>();
        ta.stats = P.stats.as<unsigned long long>();
        ta.bounce = 0;
        ta.work = P.ctr64.as<unsigned long long>();
        ta.q_out = qs[0];
        ta.q_out_count = q_count + 1;
        if (P.tune.raster) {
            ta.vis = P.vis.as<unsigned long long>();
            ta.vis_full = P.visfull.as<unsigned>();
            ta.big = P.rbig.as<int4>();
            ta.big_ctr = P.rbigctr.as<unsigned>();
            ta.big_cap = P.big_cap;
            ta.tri_pos = c->tripos.as<int>();
            ta.list_count = total_dev + 4;
            if (!ta.bistatic && !ta.wide && !ta.packet && (P.max_bounces >= 2 || escape))
                ta.hit_list = P.hitlist.as<uint2>();
            e = launch_raster(ta, (int)c->n_tri, P.vis.as<unsigned long long>(), P.visfull.as<unsigned>(), P.count,
                              c->n_sms * 16, P.scan_scr.p, st);
            if (e != cudaSuccess) break;
        } else if (P.tune.silhouette) {
            e = cudaMemsetAsync(P.cover.p, 0, sizeof(unsigned) * (size_t)(rays / 32 + na), st);
            if (e == cudaSuccess) e = launch_silhouette(ta, (int)c->n_tri, P.cover.as<unsigned>(), st);
            if (e != cudaSuccess) break;
            ta.cover = P.cover.as<unsigned>();
        }
        e = launch_trace(ta, n_blocks, P.count, P.tune.stack_depth, st);
        if (e == cudaSuccess) e = scan_popc(ta.mask, P.tilebase.as<unsigned>(), rays / 32, total_dev, P.scan_scr.p, st);
        if (e == cudaSuccess)
            e = launch_angle_offsets(ta.ray_off, ta.tile_base, total_dev, na, P.recoff.as<unsigned>(), st);
        if (e != cudaSuccess) break;
        ta.rec = P.rec.as<Record>();
        if (P.max_bounces == 1 && !escape) {
            ta.q_in = qs[0];
            ta.q_in_count = q_count + 1;
            e = launch_emit_all(ta, n_blocks, st);
        } else {
            const int last_pass = escape ? P.max_bounces : P.max_bounces - 1;
            for (int b = 1; b <= last_pass && e == cudaSuccess; ++b) {
                ta.bounce = b;
                ta.work = P.ctr64.as<unsigned long long>() + b;
                ta.q_in = qs[(b - 1) & 1];
                ta.q_in_count = q_count + b;
                ta.q_out = qs[b & 1];
                ta.q_out_count = q_count + b + 1;
                e = launch_trace(ta, n_blocks, P.count, P.tune.stack_depth, st);
                ta.hit_list = nullptr;  // only bounce pass 1 reads the list
            }
        }
        PoAngle* pang = P.pang.as<PoAngle>() + a0;
        if (e == cudaSuccess)
            e = launch_po_items(P.recoff.as<unsigned>(), pang, na, P.pa.n_pol, P.tune.po_item, P.items.as<PoItem>(),
                                P.nitems.as<int>(), P.valid.as<long long>() + k, st);
        if (e == cudaSuccess && P.items_bound[k] > 0) {
            PoArgs pa = P.pa;
            pa.rec = P.rec.as<Record>();
            pa.items = P.items.as<PoItem>();
            pa.n_items = 0;
            pa.n_items_dev = P.nitems.as<int>();
            pa.freq = P.freq_t.as<float4>();
            pa.kfreq = P.kfreq.as<double>();
            pa.partial = P.partial.as<double>();
            pa.item_records = P.tune.po_item;
            e = launch_po(pa, st, (int)std::min<long long>(P.items_bound[k], (long long)c->n_sms * 8));
        }
        if (e == cudaSuccess)
            e = launch_po_final(P.partial.as<double>(), P.items.as<PoItem>(), pang, na, P.kfreq.as<double>(),
                                P.pa.n_pol, P.E, P.R, st);
    }
    return e;
}

// Build a plan (tables uploaded, buffers sized); the graph is captured by the caller.
int build_plan(sbr_ctx* c, BatchPlan& P)
{
    const int64_t n = (int64_t)P.req.size();
    const int tw = log2i(P.tune.tile_w);
    std::vector<sbr_ray_grid> g((size_t)n);
    std::vector<long long> begin((size_t)n);
    long long total = 0;
    for (int64_t a = 0; a < n; ++a) {
        make_grid(c->bbox, P.req[(size_t)a].az_deg, P.req[(size_t)a].el_deg, P.req[(size_t)a].ray_spacing_m, P.eta,
                  &P.opt, &g[(size_t)a]);
        const long long cap = P.opt.chunk_rays > 0 ? std::max<long long>(32, P.opt.chunk_rays) : (1ll << P.tune.chunk_rays_log2);
        if (g[(size_t)a].nu > (1ll << 30) || g[(size_t)a].nv > (1ll << 30) || tiled_rays(g[(size_t)a], tw) > cap)
            return fail(c, SBR_ERR_ARG, "ray grid of request %lld too large (%lld x %lld) for a chunk of %lld rays",
                        (long long)a, (long long)g[(size_t)a].nu, (long long)g[(size_t)a].nv, cap);
        begin[(size_t)a] = total;
        total += tiled_rays(g[(size_t)a], tw);
        P.launched += g[(size_t)a].nu * g[(size_t)a].nv;
    }
    const long long cap = P.opt.chunk_rays > 0 ? std::max<long long>(32, P.opt.chunk_rays) : (1ll << P.tune.chunk_rays_log2);
    P.cut.assign(1, 0);
    long long acc = 0;
    for (int64_t a = 0; a < n; ++a) {
        const long long r = tiled_rays(g[(size_t)a], tw);
        if (acc > 0 && acc + r > cap) {
            P.cut.push_back(a);
            acc = 0;
        }
        acc += r;
    }
    P.cut.push_back(n);
    const size_t nc = P.cut.size() - 1;
    long long max_rays = 0, max_rec = 0, max_items = 0, max_part = 0;
    int max_angles = 0;
    P.chunk_rays.assign(nc, 0);
    P.items_bound.assign(nc, 0);
    for (size_t k = 0; k < nc; ++k) {
        long long rays = 0, rec = 0, items = 0, part = 0;
        for (int64_t a = P.cut[k]; a < P.cut[k + 1]; ++a) {
            const sbr_ray_grid& G = g[(size_t)a];
            rays += tiled_rays(G, tw);
            rec += G.nu * G.nv;
            const long long ni = (G.nu * G.nv + P.tune.po_item - 1) / P.tune.po_item;
            items += ni;
            part += ni * P.req[(size_t)a].n_freq * 2 * P.pa.n_pol;
        }
        P.chunk_rays[k] = rays;
        P.items_bound[k] = items;
        max_rays = std::max(max_rays, rays);
        max_rec = std::max(max_rec, rec);
        max_items = std::max(max_items, items);
        max_part = std::max(max_part, part);
        max_angles = std::max(max_angles, (int)(P.cut[k + 1] - P.cut[k]));
    }
    if (max_items >= (1ll << 31)) return fail(c, SBR_ERR_ARG, "sbr_submit_batch: chunk too large for the PO work list");
    const long long max_tiles = max_rays / 32;
    CK(P.angles.ensure(sizeof(AngleDev) * (size_t)n), "alloc angles");
    CK(P.rayoff.ensure(sizeof(long long) * (size_t)(n + nc)), "alloc ray offsets");
    CK(P.pang.ensure(sizeof(PoAngle) * (size_t)n), "alloc aspect table");
    CK(P.recoff.ensure(sizeof(unsigned) * (size_t)(max_angles + 1)), "alloc record offsets");
    CK(P.mask.ensure(sizeof(unsigned) * (size_t)max_tiles), "alloc mask");
    if (P.tune.silhouette) CK(P.cover.ensure(sizeof(unsigned) * (size_t)(max_tiles + max_angles)), "alloc cover");
    if (P.tune.raster) {
        CK(P.vis.ensure(sizeof(unsigned long long) * (size_t)max_rays), "alloc raster keys");
        CK(P.visfull.ensure(sizeof(unsigned) * (size_t)(max_angles + 1)), "alloc raster flags");
        CK(P.hitlist.ensure(sizeof(uint2) * (size_t)max_rays), "alloc raster hit list");
        P.big_cap = (unsigned)raster_big_cap(max_rays);
        CK(P.rbig.ensure(sizeof(int4) * (size_t)P.big_cap), "alloc raster triangle list");
        CK(P.rbigctr.ensure(sizeof(unsigned) * 2), "alloc raster triangle counters");
    }
    CK(P.tilebase.ensure(sizeof(unsigned) * (size_t)max_tiles), "alloc tile base");
    CK(P.scan_scr.ensure(scan_scratch_bytes(max_tiles)), "alloc scan scratch");
    CK(P.q0.ensure(sizeof(RayState) * (size_t)max_rays), "alloc ray queue");
    CK(P.q1.ensure(sizeof(RayState) * (size_t)max_rays), "alloc ray queue");
    CK(P.ctr64.ensure(sizeof(unsigned long long) * 2 * (kMaxBounces + 2)), "alloc counters");
    CK(P.ctr32.ensure(sizeof(unsigned) * 2 * (kMaxBounces + 2) + 64), "alloc counters");
    CK(P.stats.ensure(sizeof(unsigned long long) * kStatCount), "alloc stats");
    CK(P.rec.ensure(sizeof(Record) * (size_t)std::max(max_rec, 1ll)), "alloc records");
    CK(P.items.ensure(sizeof(PoItem) * (size_t)std::max(max_items, 1ll)), "alloc items");
    CK(P.nitems.ensure(sizeof(int)), "alloc item count");
    CK(P.valid.ensure(sizeof(long long) * nc), "alloc valid counts");
    CK(P.partial.ensure(sizeof(double) * (size_t)std::max(max_part, 1ll)), "alloc partials");
    CK(P.freq_t.ensure(sizeof(float4) * P.freq.size()), "alloc freq");
    CK(P.kfreq.ensure(sizeof(double) * P.freq.size()), "alloc freq");
    // tables: angles, per-chunk ray offsets, aspect rows, frequencies (one synchronous upload)
    const size_t b_a = sizeof(AngleDev) * (size_t)n, b_o = sizeof(long long) * (size_t)(n + nc),
                 b_p = sizeof(PoAngle) * (size_t)n, b_f = sizeof(float4) * P.freq.size(),
                 b_k = sizeof(double) * P.freq.size();
    char* hs = (char*)stage(c, b_a + b_o + b_p + b_f + b_k + 256);
    if (!hs) return fail(c, SBR_ERR_OOM, "pinned staging allocation failed");
    AngleDev* ha = (AngleDev*)hs;
    long long* ho = (long long*)(hs + b_a);
    PoAngle* hp = (PoAngle*)(hs + b_a + b_o);
    float4* hf = (float4*)(hs + b_a + b_o + b_p);
    double* hk = (double*)(hs + b_a + b_o + b_p + b_f);
    long long row = 0;
    for (int64_t a = 0; a < n; ++a) {
        PoAngle& A = hp[a];
        memset(&A, 0, sizeof(A));
        A.f0 = (int)P.req[(size_t)a].freq_offset;
        A.nf = P.req[(size_t)a].n_freq;
        A.out_row = row;
        row += A.nf;
    }
    for (size_t k = 0; k < nc; ++k) {
        const long long base = begin[(size_t)P.cut[k]];
        for (int64_t a = P.cut[k]; a < P.cut[k + 1]; ++a) {
            ho[a + (int64_t)k] = begin[(size_t)a] - base;
            ha[a] = to_dev(g[(size_t)a], begin[(size_t)a] - base, tw);
        }
        ho[P.cut[k + 1] + (int64_t)k] = P.chunk_rays[k];
    }
    for (size_t f = 0; f < P.freq.size(); ++f) {
        const double kappa = P.freq[f] / kC0;
        const float kh = (float)kappa;
        const double kk = 2.0 * kPi * P.freq[f] / kC0;
        hf[f] = make_float4(kh, (float)(kappa - (double)kh), (float)kk, 0.f);
        hk[f] = kk;
    }
    CK(cudaMemcpyAsync(P.angles.p, ha, b_a, cudaMemcpyHostToDevice, c->stream), "copy angles");
    CK(cudaMemcpyAsync(P.rayoff.p, ho, b_o, cudaMemcpyHostToDevice, c->stream), "copy ray offsets");
    CK(cudaMemcpyAsync(P.pang.p, hp, b_p, cudaMemcpyHostToDevice, c->stream), "copy aspect table");
    CK(cudaMemcpyAsync(P.freq_t.p, hf, b_f, cudaMemcpyHostToDevice, c->stream), "copy freq");
    CK(cudaMemcpyAsync(P.kfreq.p, hk, b_k, cudaMemcpyHostToDevice, c->stream), "copy freq");
    CK(cudaStreamSynchronize(c->stream), "plan upload sync");
    // kernels per run: stats memset excluded; per chunk trace passes, 3 scan, offsets, 2 work list, PO, final
    const bool escape = P.flags & SBR_TRACE_REQUIRE_ESCAPE;
    const int passes = (P.max_bounces == 1 && !escape) ? 1 : 1 + (escape ? P.max_bounces : P.max_bounces - 1);
    P.n_pass = (int64_t)nc * passes;
    P.n_launch = 0;
    for (size_t k = 0; k < nc; ++k)
        P.n_launch += passes + ((P.max_bounces == 1 && !escape) ? 1 : 0) + 3 + 1 + 2 + (P.items_bound[k] > 0 ? 1 : 0) + 1 +
                      (P.tune.raster ? 6 : (P.tune.silhouette ? 1 : 0));
    return SBR_OK;
}

// sbr_trace and sbr_trace_bistatic (az_el_rx: [n][2] receivers, or null for monostatic)
// ---------------------------------------------------------------- pooled late passes
// A trace of several chunks runs bounce passes 1 .. kPoolPass - 1 per chunk;
// the last of them appends the rays that go on to one pool, and passes
// kPoolPass .. run over the pool once for all chunks (a late pass holds few
// rays per chunk, and a launch over few rays leaves most SMs idle while its
// slowest rays finish). A pooled ray carries its trace-wide aspect index: the
// pooled passes read the trace's aspect table, its ray offsets, the trace-wide
// hit masks and each aspect's first record, so every record lands where the
// chunk reserved it. The pool holds as many rays as a chunk queue; rays that
// find it full stay in the chunk's queue, and at the host's next wait the pool
// is traced and they are appended.
constexpr int kPoolPass = 2;
// sbr_run_batch: a group of chunks holds the records of at most this many chunks' worth of rays
constexpr long long kGroupRecords = 4;

struct PoolRun {
    bool on = false;
    int64_t n_angles = 0;
    unsigned cap = 0;
    std::vector<long long> rec_of;  // per aspect: first record of its chunk
    // grouping of each pooled pass's rays by (aspect, triangle left >> tri_shift)
    int tri_shift = 0;
    unsigned groups = 1;
    long long n_buckets = 1;
    unsigned* counts = nullptr;
    unsigned* order = nullptr;
    void* scan_scratch = nullptr;
};
constexpr long long kMaxBuckets = 1ll << 22;

// run the pooled passes over the pool (its ping-pong partner: queue `partner`), then empty it
int flush_pool(sbr_ctx* c, TraceRun& R, PoolRun& P, RayState* partner)
{
    const int last_pass = R.escape ? R.max_bounces : R.max_bounces - 1;
    const size_t b_rec = sizeof(long long) * (size_t)P.n_angles;
    long long* hr = (long long*)stage(c, b_rec);
    if (!hr) return fail(c, SBR_ERR_OOM, "pinned staging allocation failed");
    memcpy(hr, P.rec_of.data(), b_rec);
    CK(cudaMemcpyAsync(c->recofall.p, hr, b_rec, cudaMemcpyHostToDevice, c->stream), "copy record bases");
    CK(cudaEventRecord(c->stage_ev, c->stream), "record staging event");
    unsigned* ctr = c->poolctr.as<unsigned>();  // [0] pool count, [1] flag, [2 + j] output of pooled pass j
    CK(cudaMemsetAsync(ctr + 2, 0, sizeof(unsigned) * (kMaxBounces + 2), c->stream), "memset pool counters");
    CK(cudaMemsetAsync(c->poolwork.p, 0, c->poolwork.cap, c->stream), "memset pool work");
    TraceArgs ta;
    memset(&ta, 0, sizeof(ta));
    ta.wide = c->tune.bvh_width == 4;
    ta.packet = c->tune.packet;
    ta.octant = c->tune.octant;
    ta.n_nodes = c->n_nodes;
    for (int64_t a = 0; a < P.n_angles; ++a) ta.bistatic |= c->ang[(size_t)a].bistatic ? 1 : 0;
    if (ta.octant) CK(ensure_octant_nodes(c, c->stream), "octant nodes");
    ta.nodes = ta.wide ? c->nodes4.as<float4>() : (ta.octant ? c->nodes_oct.as<float4>() : c->nodes.as<float4>());
    ta.tris = c->tris.as<float4>();
    ta.tri_nrm = ta.tris + 3 * (size_t)c->n_tri;
    ta.tri_v12 = ta.tris + 4 * (size_t)c->n_tri;
    ta.angles = c->angall.as<AngleDev>();
    ta.ray_off = c->rayoffall.as<long long>();
    ta.n_angles = (int)P.n_angles;
    ta.max_bounces = R.max_bounces;
    ta.flags = R.flags;
    ta.visit_limit = (int)std::min<long long>(2 * c->n_tri + 64, 1ll << 30);
    ta.mask = c->mask.as<unsigned>();
    ta.tile_base = c->tilebase.as<unsigned>();
    ta.stats = c->stats.as<unsigned long long>();
    ta.rec = c->rec.as<Record>();
    ta.rec_of = c->recofall.as<long long>();
    if (R.hits) {
        ta.hit_tri = c->hit_tri.as<int>();
        ta.hit_t = c->hit_t.as<float>();
        ta.hit_nb = c->hit_nb.as<int>();
    }
    RayState* qs[2] = {c->pool.as<RayState>(), partner};
    for (int b = kPoolPass; b <= last_pass; ++b) {
        const int j = b - kPoolPass;
        ta.bounce = b;
        ta.work = c->poolwork.as<unsigned long long>() + j;
        ta.q_in = qs[j & 1];
        ta.q_in_count = j == 0 ? ctr : ctr + 2 + (j - 1);
        ta.q_out = qs[(j + 1) & 1];
        ta.q_out_count = ctr + 2 + j;
        // the pass takes its rays grouped by aspect and by the triangle they leave
        CK(cudaMemsetAsync(P.counts, 0, sizeof(unsigned) * (size_t)P.n_buckets, c->stream), "memset buckets");
        CK(launch_group_rays(ta.q_in, ta.q_in_count, P.tri_shift, P.groups, P.counts, P.n_buckets, P.order,
                             P.scan_scratch, c->n_sms * 4, c->stream),
           "group rays");
        R.n_launch += 5;
        ta.q_order = P.order;
        CK(run_pass(c, R, ta), "trace pooled pass");
    }
    CK(cudaMemsetAsync(ctr, 0, sizeof(unsigned) * 2, c->stream), "memset pool count");
    return SBR_OK;
}

// after a chunk: copy the pool's count and flag, and the count of the chunk's rays that found the pool full, to
// c->pool_host (pinned) for the host's next wait
int pool_note(sbr_ctx* c)
{
    const int b = kPoolPass - 1;  // the chunk's last pass: its overflow count at q_count + b + 1
    CK(cudaMemcpyAsync(c->pool_host, c->poolctr.p, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream),
       "copy pool count");
    CK(cudaMemcpyAsync(c->pool_host + 2, c->ctr32.as<unsigned>() + b + 1, sizeof(unsigned), cudaMemcpyDeviceToHost,
                       c->stream),
       "copy pool overflow");
    return SBR_OK;
}

// after the wait that follows a chunk whose rays did not all fit the pool: trace the full pool, then append the
// rays the chunk kept in its queue (their aspect index already the trace's)
int pool_overflow(sbr_ctx* c, TraceRun& R, PoolRun& P, RayState* partner)
{
    const int b = kPoolPass - 1;
    RayState* qs[2] = {c->q0.as<RayState>(), c->q1.as<RayState>()};
    unsigned* ctr = c->poolctr.as<unsigned>();
    c->pool_host[3] = P.cap;
    CK(cudaMemcpyAsync(ctr, c->pool_host + 3, sizeof(unsigned), cudaMemcpyHostToDevice, c->stream), "set pool count");
    int r = flush_pool(c, R, P, partner);
    if (r != SBR_OK) return r;
    CK(launch_pool_append(qs[b & 1], c->ctr32.as<unsigned>() + b + 1, c->pool.as<RayState>(), ctr, P.cap, 0, ctr + 1,
                          c->n_sms * 4, c->stream),
       "pool append");
    R.n_launch += 2;
    r = pool_note(c);
    if (r != SBR_OK) return r;
    CK(cudaStreamSynchronize(c->stream), "pool sync");
    return c->pool_host[1] ? fail(c, SBR_ERR_STATE, "sbr_trace: a chunk's live rays do not fit the ray pool") : SBR_OK;
}

// set up the pool for a trace of the chunks cut (aspects c->ang, grids and ray offsets planned)
int pool_setup(sbr_ctx* c, TraceRun& R, PoolRun& P, const std::vector<int64_t>& cut)
{
    const int64_t n = (int64_t)c->ang.size();
    const int last_pass = R.escape ? R.max_bounces : R.max_bounces - 1;
    P.on = cut.size() > 2 && last_pass >= kPoolPass && n <= (1 << 20);
    if (!P.on) return SBR_OK;
    P.n_angles = n;
    P.cap = (unsigned)std::min<size_t>(c->q0.cap / sizeof(RayState), 0xFFFFFFFFu);
    P.rec_of.assign((size_t)n, 0);
    CK(c->pool.ensure(sizeof(RayState) * (size_t)P.cap), "alloc ray pool");
    CK(c->angall.ensure(sizeof(AngleDev) * (size_t)n), "alloc aspect table");
    CK(c->rayoffall.ensure(sizeof(long long) * (size_t)(n + 1)), "alloc ray offsets");
    CK(c->recofall.ensure(sizeof(long long) * (size_t)n), "alloc record bases");
    CK(c->poolctr.ensure(sizeof(unsigned) * (kMaxBounces + 4)), "alloc pool counters");
    CK(c->poolwork.ensure(sizeof(unsigned long long) * (kMaxBounces + 2)), "alloc pool work counters");
    while (P.tri_shift < 30) {
        P.groups = (unsigned)((c->n_tri + (1ll << P.tri_shift) - 1) >> P.tri_shift);
        if ((long long)P.groups * n <= kMaxBuckets) break;
        ++P.tri_shift;
    }
    P.n_buckets = std::max(1ll, (long long)P.groups * n);
    {
        const size_t b_cnt = ((sizeof(unsigned) * (size_t)P.n_buckets + 255) / 256) * 256;
        const size_t b_ord = ((sizeof(unsigned) * (size_t)P.cap + 255) / 256) * 256;
        CK(c->poolgroup.ensure(b_cnt + b_ord + scan_scratch_bytes(P.n_buckets)), "alloc ray grouping");
        char* g = (char*)c->poolgroup.p;
        P.counts = (unsigned*)g;
        P.order = (unsigned*)(g + b_cnt);
        P.scan_scratch = g + b_cnt + b_ord;
    }
    if (!c->pool_host && cudaMallocHost((void**)&c->pool_host, 4 * sizeof(unsigned)) != cudaSuccess) {
        c->pool_host = nullptr;
        return fail(c, SBR_ERR_OOM, "pinned allocation failed");
    }
    const size_t b_a = sizeof(AngleDev) * (size_t)n, b_o = sizeof(long long) * (size_t)(n + 1);
    char* hs = (char*)stage(c, b_a + b_o);
    if (!hs) return fail(c, SBR_ERR_OOM, "pinned staging allocation failed");
    AngleDev* ha = (AngleDev*)hs;
    long long* ho = (long long*)(hs + b_a);
    for (int64_t a = 0; a < n; ++a) {
        const AngleHost& h = c->ang[(size_t)a];
        ho[a] = h.ray_begin;
        double rx[2] = {h.rx_az, h.rx_el};
        ha[a] = to_dev(h.grid, h.ray_begin, h.tw, h.bistatic ? rx : nullptr);
    }
    const AngleHost& l = c->ang[(size_t)n - 1];
    ho[n] = l.ray_begin + tiled_rays(l.grid, l.tw);
    CK(cudaMemcpyAsync(c->angall.p, ha, b_a, cudaMemcpyHostToDevice, c->stream), "copy aspect table");
    CK(cudaMemcpyAsync(c->rayoffall.p, ho, b_o, cudaMemcpyHostToDevice, c->stream), "copy ray offsets");
    CK(cudaMemsetAsync(c->poolctr.p, 0, c->poolctr.cap, c->stream), "memset pool counters");
    CK(cudaEventRecord(c->stage_ev, c->stream), "record staging event");
    R.stop_after = kPoolPass - 1;
    R.pool = c->pool.as<RayState>();
    R.pool_count = c->poolctr.as<unsigned>();
    R.pool_cap = P.cap;
    return SBR_OK;
}

int trace_impl(sbr_ctx* c, const double* az_el, const double* az_el_rx, int64_t n_angles, double ds, double eta,
               int max_bounces, const sbr_trace_opts* opt, sbr_trace_stats* stats)
{
    if (!c) return SBR_ERR_ARG;
    if (!c->has_bvh) return fail(c, SBR_ERR_STATE, "sbr_trace: no BVH (load a mesh first)");
    if (!az_el || n_angles < 1) return fail(c, SBR_ERR_ARG, "sbr_trace: no angles");
    if (n_angles > (1ll << 30)) return fail(c, SBR_ERR_ARG, "sbr_trace: too many angles");
    if (!(ds > 0.0) || !(eta >= 0.0)) return fail(c, SBR_ERR_ARG, "sbr_trace: spacing must be > 0, eta >= 0");
    if (max_bounces < 1 || max_bounces > kMaxBounces) return fail(c, SBR_ERR_ARG, "sbr_trace: max_bounces in 1..128");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    TraceRun R;
    R.flags = opt ? opt->flags : 0;
    R.max_bounces = max_bounces;
    R.escape = R.flags & SBR_TRACE_REQUIRE_ESCAPE;
    R.hits = R.flags & SBR_TRACE_RECORD_HITS;
    R.count = R.flags & SBR_TRACE_COUNT_VISITS;
    R.timed = R.flags & SBR_TRACE_TIME_PASSES;
    R.chunk_cap = (opt && opt->chunk_rays > 0) ? std::max<long long>(32, opt->chunk_rays)
                                                : (1ll << c->tune.chunk_rays_log2);
    c->has_trace = false;
    c->ang.resize((size_t)n_angles);
    for (int64_t a = 0; a < n_angles; ++a) {
        AngleHost& h = c->ang[(size_t)a];
        make_grid(c->bbox, az_el[2 * a], az_el[2 * a + 1], ds, eta, opt, &h.grid);
        h.tw = log2i(c->tune.tile_w);
        h.bistatic = az_el_rx != nullptr;
        h.rx_az = az_el_rx ? az_el_rx[2 * a] : 0.0;
        h.rx_el = az_el_rx ? az_el_rx[2 * a + 1] : 0.0;
    }
    std::vector<int64_t> cut;
    long long total = 0, launched = 0;
    int rc = plan_chunks(c, R, cut, &total, &launched);
    if (rc != SBR_OK) return rc;
    c->rec_total = 0;
    PoolRun P;
    rc = pool_setup(c, R, P, cut);
    if (rc != SBR_OK) return rc;
    RayState* partner = c->q0.as<RayState>();  // the chunk queue free between chunks (kPoolPass - 1 wrote q1)
    static_assert(kPoolPass == 2, "the pool's partner queue assumes the chunks stop after bounce pass 1");
    // the host waits once per chunk: a chunk's records start where the previous chunk's end; rays that found
    // the pool full are appended once it has been traced
    unsigned* hro = nullptr;
    auto settle = [&]() -> int {  // after the wait that follows a chunk
        if (!P.on || c->pool_host[0] <= P.cap) return SBR_OK;
        return pool_overflow(c, R, P, partner);
    };
    for (size_t k = 0; k + 1 < cut.size(); ++k) {
        if (k > 0) {
            CK(cudaStreamSynchronize(c->stream), "trace sync");
            c->rec_total += chunk_records(c, cut[k - 1], cut[k], c->rec_total, hro);
            rc = settle();
            if (rc != SBR_OK) return rc;
        }
        if (P.on)
            for (int64_t a = cut[k]; a < cut[k + 1]; ++a) P.rec_of[(size_t)a] = c->rec_total;
        rc = trace_chunk(c, R, cut[k], cut[k + 1], c->rec_total, &hro);
        if (rc == SBR_OK && P.on) rc = pool_note(c);
        if (rc != SBR_OK) return rc;
    }
    if (P.on) {
        CK(cudaStreamSynchronize(c->stream), "trace sync");
        rc = settle();
        if (rc == SBR_OK) rc = flush_pool(c, R, P, partner);
        if (rc != SBR_OK) return rc;
    }
    unsigned long long hs_stats[kStatCount];
    rc = read_counters(c, hs_stats);
    if (rc != SBR_OK) return rc;
    const size_t last = cut.size() - 2;
    c->rec_total += chunk_records(c, cut[last], cut[last + 1], c->rec_total, hro);
    rc = finish_stats(c, R, hs_stats, n_angles, launched, c->rec_total, stats);
    c->max_bounces = max_bounces;
    c->trace_flags = R.flags;
    c->has_trace = rc == SBR_OK;
    return rc;
}

}  // namespace

extern "C" {

int sbr_trace(sbr_ctx* c, const double* az_el, int64_t n_angles, double ds, double eta, int max_bounces,
              const sbr_trace_opts* opt, sbr_trace_stats* stats)
{
    return trace_impl(c, az_el, nullptr, n_angles, ds, eta, max_bounces, opt, stats);
}

int sbr_trace_bistatic(sbr_ctx* c, const double* az_el_tx, const double* az_el_rx, int64_t n_angles, double ds,
                       double eta, int max_bounces, const sbr_trace_opts* opt, sbr_trace_stats* stats)
{
    if (c && !az_el_rx) return fail(c, SBR_ERR_ARG, "sbr_trace_bistatic: no receiver angles");
    return trace_impl(c, az_el_tx, az_el_rx, n_angles, ds, eta, max_bounces, opt, stats);
}

int sbr_po_integrate(sbr_ctx* c, const double* freq_hz, int64_t n_freq, int pol_mask, int po_mode, double* E_out,
                     double* rcs_out, int out_on_device)
{
    if (!c) return SBR_ERR_ARG;
    if (!c->has_trace) return fail(c, SBR_ERR_STATE, "sbr_po_integrate: no trace results");
    if (!freq_hz || n_freq < 1 || n_freq > (1 << 20)) return fail(c, SBR_ERR_ARG, "sbr_po_integrate: bad frequency list");
    PoArgs pa;
    int rc = check_po_mode(c, pol_mask, po_mode, pa);
    if (rc != SBR_OK) return rc;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    rc = upload_freqs(c, freq_hz, n_freq);
    if (rc != SBR_OK) return rc;
    pa.n_freq = (int)n_freq;
    const int64_t na = (int64_t)c->ang.size();
    std::vector<int> f0((size_t)na, 0), nf((size_t)na, (int)n_freq);
    std::vector<long long> row((size_t)na);
    for (int64_t a = 0; a < na; ++a) row[(size_t)a] = a * n_freq;
    const size_t n_out = (size_t)na * (size_t)n_freq * pa.n_pol;
    double* dE = E_out;
    double* dR = rcs_out;
    if (!out_on_device) {
        CK(c->E.ensure(sizeof(double) * 2 * n_out), "alloc E");
        CK(c->rcs.ensure(sizeof(double) * n_out), "alloc rcs");
        dE = E_out ? c->E.as<double>() : nullptr;
        dR = rcs_out ? c->rcs.as<double>() : nullptr;
    }
    CK(cudaMemsetAsync(c->err_dev.as<int>() + 3, 0, sizeof(int), c->stream), "memset po flag");
    rc = po_run(c, pa, 0, na, f0, nf, row, dE, dR, nullptr);
    if (rc != SBR_OK) return rc;
    if (!out_on_device) {
        int flag = 0;
        if (E_out)
            CK(cudaMemcpyAsync(E_out, dE, sizeof(double) * 2 * n_out, cudaMemcpyDeviceToHost, c->stream), "copy E");
        if (rcs_out)
            CK(cudaMemcpyAsync(rcs_out, dR, sizeof(double) * n_out, cudaMemcpyDeviceToHost, c->stream), "copy rcs");
        CK(cudaMemcpyAsync(&flag, c->err_dev.as<int>() + 3, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
           "copy po flag");
        CK(cudaStreamSynchronize(c->stream), "po sync");
        if (flag) return fail(c, SBR_ERR_TIMEOUT, "sbr_po_integrate: a staged record load did not arrive");
    }
    return SBR_OK;
}

int sbr_run_batch(sbr_ctx* c, const sbr_request* req, int64_t n_req, const double* freq_hz, int64_t n_freq_total,
                  double eta, int max_bounces, int pol_mask, int po_mode, const sbr_trace_opts* opt, double* E_out,
                  double* rcs_out, int out_on_device, sbr_trace_stats* stats)
{
    if (!c) return SBR_ERR_ARG;
    if (!c->has_bvh) return fail(c, SBR_ERR_STATE, "sbr_run_batch: no BVH (load a mesh first)");
    if (!req || n_req < 1 || n_req > (1ll << 30)) return fail(c, SBR_ERR_ARG, "sbr_run_batch: no requests");
    if (!freq_hz || n_freq_total < 1 || n_freq_total > (1ll << 30))
        return fail(c, SBR_ERR_ARG, "sbr_run_batch: bad frequency array");
    if (!(eta >= 0.0)) return fail(c, SBR_ERR_ARG, "sbr_run_batch: eta >= 0");
    if (max_bounces < 1 || max_bounces > kMaxBounces) return fail(c, SBR_ERR_ARG, "sbr_run_batch: max_bounces in 1..128");
    if (opt && (opt->flags & SBR_TRACE_RECORD_HITS))
        return fail(c, SBR_ERR_ARG, "sbr_run_batch: SBR_TRACE_RECORD_HITS is for sbr_trace");
    PoArgs pa;
    int rc = check_po_mode(c, pol_mask, po_mode, pa);
    if (rc != SBR_OK) return rc;
    std::vector<int> f0((size_t)n_req), nf((size_t)n_req);
    std::vector<long long> row((size_t)n_req);
    long long rows = 0;
    for (int64_t r = 0; r < n_req; ++r) {
        const sbr_request& q = req[r];
        if (!(q.ray_spacing_m > 0.0)) return fail(c, SBR_ERR_ARG, "sbr_run_batch: request %lld: spacing must be > 0", (long long)r);
        if (q.n_freq < 1 || q.freq_offset < 0 || q.freq_offset + q.n_freq > n_freq_total)
            return fail(c, SBR_ERR_ARG, "sbr_run_batch: request %lld: frequency range outside the array", (long long)r);
        f0[(size_t)r] = (int)q.freq_offset;
        nf[(size_t)r] = q.n_freq;
        row[(size_t)r] = rows;
        rows += q.n_freq;
    }
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    TraceRun R;
    R.flags = opt ? opt->flags : 0;
    R.max_bounces = max_bounces;
    R.escape = R.flags & SBR_TRACE_REQUIRE_ESCAPE;
    R.count = R.flags & SBR_TRACE_COUNT_VISITS;
    R.timed = R.flags & SBR_TRACE_TIME_PASSES;
    R.chunk_cap = (opt && opt->chunk_rays > 0) ? std::max<long long>(32, opt->chunk_rays)
                                                : (1ll << c->tune.chunk_rays_log2);
    c->has_trace = false;
    c->ang.resize((size_t)n_req);
    for (int64_t r = 0; r < n_req; ++r) {
        make_grid(c->bbox, req[r].az_deg, req[r].el_deg, req[r].ray_spacing_m, eta, opt, &c->ang[(size_t)r].grid);
        c->ang[(size_t)r].tw = log2i(c->tune.tile_w);
        c->ang[(size_t)r].bistatic = false;
    }
    std::vector<int64_t> cut;
    long long total = 0, launched = 0;
    rc = plan_chunks(c, R, cut, &total, &launched);
    if (rc != SBR_OK) return rc;
    rc = upload_freqs(c, freq_hz, n_freq_total);
    if (rc != SBR_OK) return rc;
    pa.n_freq = (int)n_freq_total;
    const size_t n_out = (size_t)rows * pa.n_pol;
    double* dE = E_out;
    double* dR = rcs_out;
    if (!out_on_device) {
        CK(c->E.ensure(sizeof(double) * 2 * n_out), "alloc E");
        CK(c->rcs.ensure(sizeof(double) * n_out), "alloc rcs");
        dE = E_out ? c->E.as<double>() : nullptr;
        dR = rcs_out ? c->rcs.as<double>() : nullptr;
    }
    // each chunk is traced once and integrated for all its requests' frequencies. Without the ray pool every
    // chunk is integrated before the next reuses the record buffer; with it, consecutive chunks form a group whose
    // records stay until the group's pooled late passes have run, and the group is integrated then
    long long valid = 0, rec_base = 0;
    size_t g0 = 0;
    CK(cudaMemsetAsync(c->err_dev.as<int>() + 3, 0, sizeof(int), c->stream), "memset po flag");
    PoolRun P;
    rc = pool_setup(c, R, P, cut);
    if (rc != SBR_OK) return rc;
    RayState* partner = c->q0.as<RayState>();
    auto close_group = [&](size_t g1) -> int {
        int r = flush_pool(c, R, P, partner);
        if (r == SBR_OK) r = po_run(c, pa, cut[g0], cut[g1], f0, nf, row, dE, dR, &R.n_launch);
        rec_base = 0;
        g0 = g1;
        return r;
    };
    for (size_t k = 0; k + 1 < cut.size(); ++k) {
        const AngleHost& last = c->ang[(size_t)cut[k + 1] - 1];
        const long long rays = last.ray_begin + tiled_rays(last.grid, last.tw) - c->ang[(size_t)cut[k]].ray_begin;
        if (P.on && k > g0 && rec_base + rays > kGroupRecords * R.chunk_cap) {
            rc = close_group(k);
            if (rc != SBR_OK) return rc;
        }
        if (P.on)
            for (int64_t a = cut[k]; a < cut[k + 1]; ++a) P.rec_of[(size_t)a] = rec_base;
        unsigned* hro = nullptr;
        rc = trace_chunk(c, R, cut[k], cut[k + 1], rec_base, &hro);
        if (rc == SBR_OK && P.on) rc = pool_note(c);
        if (rc != SBR_OK) return rc;
        CK(cudaStreamSynchronize(c->stream), "trace sync");
        const long long n = chunk_records(c, cut[k], cut[k + 1], rec_base, hro);
        valid += n;
        if (P.on) {
            rec_base += n;
            if (c->pool_host[0] > P.cap) rc = pool_overflow(c, R, P, partner);
        } else {
            rc = po_run(c, pa, cut[k], cut[k + 1], f0, nf, row, dE, dR, &R.n_launch);
        }
        if (rc != SBR_OK) return rc;
    }
    if (P.on) {
        rc = close_group(cut.size() - 1);
        if (rc != SBR_OK) return rc;
    }
    if (!out_on_device) {
        if (E_out)
            CK(cudaMemcpyAsync(E_out, dE, sizeof(double) * 2 * n_out, cudaMemcpyDeviceToHost, c->stream), "copy E");
        if (rcs_out)
            CK(cudaMemcpyAsync(rcs_out, dR, sizeof(double) * n_out, cudaMemcpyDeviceToHost, c->stream), "copy rcs");
    }
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, c->err_dev.as<int>() + 3, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
       "copy po flag");
    unsigned long long hs_stats[kStatCount];
    rc = read_counters(c, hs_stats);  // synchronises the stream
    if (rc != SBR_OK) return rc;
    if (flag) return fail(c, SBR_ERR_TIMEOUT, "sbr_run_batch: a staged record load did not arrive");
    return finish_stats(c, R, hs_stats, n_req, launched, valid, stats);
}

int sbr_submit_batch(sbr_ctx* c, const sbr_request* req, int64_t n_req, const double* freq_hz, int64_t n_freq_total,
                     double eta, int max_bounces, int pol_mask, int po_mode, const sbr_trace_opts* opt, double* E_dev,
                     double* rcs_dev)
{
    if (!c) return SBR_ERR_ARG;
    if (!c->has_bvh) return fail(c, SBR_ERR_STATE, "sbr_submit_batch: no BVH (load a mesh first)");
    if (!req || n_req < 1 || n_req > (1ll << 30)) return fail(c, SBR_ERR_ARG, "sbr_submit_batch: no requests");
    if (!freq_hz || n_freq_total < 1 || n_freq_total > (1ll << 30))
        return fail(c, SBR_ERR_ARG, "sbr_submit_batch: bad frequency array");
    if (!(eta >= 0.0)) return fail(c, SBR_ERR_ARG, "sbr_submit_batch: eta >= 0");
    if (max_bounces < 1 || max_bounces > kMaxBounces)
        return fail(c, SBR_ERR_ARG, "sbr_submit_batch: max_bounces in 1..128");
    sbr_trace_opts o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    if (o.flags & (SBR_TRACE_RECORD_HITS | SBR_TRACE_TIME_PASSES))
        return fail(c, SBR_ERR_ARG, "sbr_submit_batch: SBR_TRACE_RECORD_HITS / SBR_TRACE_TIME_PASSES are refused");
    for (int64_t f = 0; f < n_freq_total; ++f)
        if (!(freq_hz[f] > 0.0)) return fail(c, SBR_ERR_ARG, "sbr_submit_batch: frequencies must be > 0");
    for (int64_t r = 0; r < n_req; ++r) {
        const sbr_request& q = req[r];
        if (!(q.ray_spacing_m > 0.0))
            return fail(c, SBR_ERR_ARG, "sbr_submit_batch: request %lld: spacing must be > 0", (long long)r);
        if (q.n_freq < 1 || q.freq_offset < 0 || q.freq_offset + q.n_freq > n_freq_total)
            return fail(c, SBR_ERR_ARG, "sbr_submit_batch: request %lld: frequency range outside the array",
                        (long long)r);
    }
    PoArgs pa;
    int rc = check_po_mode(c, pol_mask, po_mode, pa);
    if (rc != SBR_OK) return rc;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    const bool graph = !(o.flags & SBR_TRACE_NO_GRAPH);
    o.flags &= ~SBR_TRACE_NO_GRAPH;
    if (!(c->plan && same_submission(*c->plan, c, req, n_req, freq_hz, n_freq_total, eta, max_bounces, pol_mask,
                                     po_mode, o, E_dev, rcs_dev))) {
        if (c->plan) CK(cudaStreamSynchronize(c->stream), "wait for the previous batch");
        free_plan(c->plan);
        c->plan = nullptr;
        c->plan_pending = false;
        BatchPlan* P = new BatchPlan();
        P->req.assign(req, req + n_req);
        P->freq.assign(freq_hz, freq_hz + n_freq_total);
        P->eta = eta;
        P->max_bounces = max_bounces;
        P->pol_mask = pol_mask;
        P->po_mode = po_mode;
        P->opt = o;
        P->flags = o.flags;
        P->count = o.flags & SBR_TRACE_COUNT_VISITS;
        P->tune = c->tune;
        P->E = E_dev;
        P->R = rcs_dev;
        P->mesh_gen = c->mesh_gen;
        P->pa = pa;
        rc = build_plan(c, *P);
        if (rc != SBR_OK) {
            free_plan(P);
            return rc;
        }
        c->plan = P;
    }
    BatchPlan& P = *c->plan;
    if (P.tune.octant) CK(ensure_octant_nodes(c, c->stream), "octant nodes");
    if (!graph) {
        CK(enqueue_plan(c, P, c->stream), "enqueue batch");
    } else {
        if (!P.exec) {
            if (!P.cap) CK(cudaStreamCreateWithFlags(&P.cap, cudaStreamNonBlocking), "capture stream");
            CK(cudaStreamBeginCapture(P.cap, cudaStreamCaptureModeThreadLocal), "begin capture");
            cudaError_t e = enqueue_plan(c, P, P.cap);
            cudaGraph_t gr = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(P.cap, &gr);
            if (e == cudaSuccess) e = e2;
            if (e != cudaSuccess) {
                if (gr) cudaGraphDestroy(gr);
                cudaGetLastError();
                return cuda_fail(c, e, "capture batch graph");
            }
            P.graph = gr;
            CK(cudaGraphInstantiate(&P.exec, P.graph, 0), "instantiate batch graph");
        }
        CK(cudaGraphLaunch(P.exec, c->stream), "launch batch graph");
    }
    c->plan_pending = true;
    return SBR_OK;
}

int sbr_sync(sbr_ctx* c, sbr_trace_stats* stats)
{
    if (!c) return SBR_ERR_ARG;
    if (!c->plan || !c->plan_pending) return fail(c, SBR_ERR_STATE, "sbr_sync: no submitted batch");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    BatchPlan& P = *c->plan;
    const size_t nc = P.cut.size() - 1;
    unsigned long long hs[kStatCount];
    std::vector<long long> hv(nc);
    CK(cudaStreamSynchronize(c->stream), "batch sync");
    CK(cudaMemcpy(hs, P.stats.p, sizeof(hs), cudaMemcpyDeviceToHost), "copy stats");
    CK(cudaMemcpy(hv.data(), P.valid.p, sizeof(long long) * nc, cudaMemcpyDeviceToHost), "copy valid counts");
    c->plan_pending = false;
    long long valid = 0;
    for (long long v : hv) valid += v;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->n_angles = (int64_t)P.req.size();
        stats->rays_launched = P.launched;
        stats->ray_bounces = (int64_t)hs[kStatQueries];
        stats->valid_rays = valid;
        stats->node_visits = (int64_t)hs[kStatNodes];
        stats->tri_tests = (int64_t)hs[kStatTris];
        stats->raster_tests = (int64_t)hs[kStatRaster];
        stats->bounce_hits = (int64_t)hs[kStatHits];
        stats->listed_hits = (int64_t)hs[kStatListed];
        stats->open_tests = (int64_t)hs[kStatOpen];
        stats->fp64_tests = (int64_t)hs[kStatFp64];
        stats->warp_node_visits = (int64_t)hs[kStatWarpNodes];
        stats->stack_overflows = (int64_t)hs[kStatOverflow];
        stats->kernel_launches = P.n_launch;
        stats->pass_launches = P.n_pass;
    }
    if (hs[kStatOverflow])
        return fail(c, SBR_ERR_STACK_OVERFLOW, "%llu traversals exceeded the stack depth",
                    (unsigned long long)hs[kStatOverflow]);
    return SBR_OK;
}

int sbr_get_tuning(const sbr_ctx* c, sbr_tuning* out)
{
    if (!c || !out) return SBR_ERR_ARG;
    *out = c->tune;
    return SBR_OK;
}

int sbr_set_tuning(sbr_ctx* c, const sbr_tuning* t)
{
    if (!c || !t) return SBR_ERR_ARG;
    if (!tuning_ok(*t)) return fail(c, SBR_ERR_ARG, "sbr_set_tuning: value out of range");
    c->tune = *t;
    return SBR_OK;
}

int sbr_autotune(sbr_ctx* c, const sbr_request* req, int64_t n_req, const double* freq_hz, int64_t n_freq_total,
                 double eta, int max_bounces, int pol_mask, int po_mode, const sbr_trace_opts* opt, int reps,
                 sbr_tune_trial* trials, int trial_cap, int* n_trials, sbr_tuning* best, double* best_ms)
{
    if (!c) return SBR_ERR_ARG;
    if (!req || n_req < 1 || !freq_hz || n_freq_total < 1 || pol_mask <= 0 || pol_mask > 15)
        return fail(c, SBR_ERR_ARG, "sbr_autotune: empty sample batch");
    if (n_trials) *n_trials = 0;
    reps = std::max(1, std::min(reps, 100));
    int n_pol = 0;
    for (int q = 0; q < 4; ++q) n_pol += (pol_mask >> q) & 1;
    long long rows = 0;
    for (int64_t r = 0; r < n_req; ++r) rows += std::max(0, req[r].n_freq);
    DevBuf dR;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    CK(dR.ensure(sizeof(double) * (size_t)std::max(1ll, rows * n_pol)), "alloc autotune output");
    const sbr_tuning start = c->tune;
    std::vector<double> ref((size_t)(rows * n_pol)), cur(ref.size());
    int nt = 0;
    // one run of the sample under setting t (results left in dR), its wall time in *ms
    auto once = [&](const sbr_tuning& t, double* ms) -> int {
        c->tune = t;
        const auto t0 = std::chrono::steady_clock::now();
        int rc = sbr_run_batch(c, req, n_req, freq_hz, n_freq_total, eta, max_bounces, pol_mask, po_mode, opt,
                               nullptr, dR.as<double>(), 1, nullptr);
        if (cudaDeviceSynchronize() != cudaSuccess) return fail(c, SBR_ERR_CUDA, "sbr_autotune: sync");
        *ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        return rc;
    };
    // a warm-up run of t (its dBsm into rcs), then `reps` timed runs of t, each followed by a run of the
    // setting `base` when given, so that both see the same drift of clocks and host; the fastest run of
    // each (host jitter only ever adds time)
    auto run = [&](const sbr_tuning& t, std::vector<double>& rcs, double* ms, const sbr_tuning* base,
                   double* base_ms) -> int {
        double w = 0.0;
        int rc = once(t, &w);
        if (rc != SBR_OK) return rc;
        if (cudaMemcpy(rcs.data(), dR.p, sizeof(double) * rcs.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(c, SBR_ERR_CUDA, "sbr_autotune: copy results");
        double fastest = 1e300, fastest_b = 1e300;
        for (int k = 0; k < reps && rc == SBR_OK; ++k) {
            rc = once(t, &w);
            fastest = std::min(fastest, w);
            if (base && rc == SBR_OK) {
                const int rb = once(*base, &w);
                if (rb != SBR_OK) return rb;
                fastest_b = std::min(fastest_b, w);
            }
        }
        *ms = fastest;
        if (base_ms) *base_ms = fastest_b;
        return rc;
    };
    auto note = [&](const sbr_tuning& t, double ms, int status) {
        if (trials && nt < trial_cap) {
            trials[nt].tuning = t;
            trials[nt].ms = ms;
            trials[nt].status = status;
            trials[nt].reserved = 0;
        }
        ++nt;
    };
    double cur_ms = 0.0;
    int rc = run(start, ref, &cur_ms, nullptr, nullptr);
    note(start, cur_ms, rc);
    if (rc != SBR_OK) {
        c->tune = start;
        if (n_trials) *n_trials = nt;
        return rc;
    }
    sbr_tuning bestt = start;
    const int occ = std::min(4, std::max(1, trace_blocks_per_sm()));
    // parameter 0 is the traversal: binary per lane, 4-wide per lane, binary per warp, binary over octant copies
    for (int p = 0; p < 8; ++p) {
        std::vector<int> vals;
        if (p == 0) vals = {0, 1, 2, 3};
        if (p == 6 || p == 7) vals = {0, 1};
        if (p == 1)
            for (int v = 1; v <= occ; ++v) vals.push_back(v);
        if (p == 2) vals = {32, 16, 8, 4};
        if (p == 3) vals = {32, 64, 128};
        if (p == 4) vals = {512, 1024, 2048};
        if (p == 5) vals = {22, 24, 25, 26, 27, 28};
        for (int v : vals) {
            sbr_tuning t = bestt;
            if (p == 0) {
                const int w = v == 1 ? 4 : 2, pk = v == 2 ? 1 : 0, oc = v == 3 ? 1 : 0;
                if (t.bvh_width == w && t.packet == pk && t.octant == oc) continue;
                t.bvh_width = w;
                t.packet = pk;
                t.octant = oc;
                if (pk && t.stack_depth > 64) t.stack_depth = 64;
            } else {
                int* fields[8] = {nullptr,    &t.blocks_per_sm,   &t.tile_w,     &t.stack_depth,
                                  &t.po_item, &t.chunk_rays_log2, &t.silhouette, &t.raster};
                if (*fields[p] == v) continue;
                *fields[p] = v;
            }
            if (!tuning_ok(t)) continue;
            double ms = 0.0, base_ms = 0.0;
            int st = run(t, cur, &ms, &bestt, &base_ms);
            if (st == SBR_OK) {
                for (size_t i = 0; i < ref.size(); ++i)
                    if (ref[i] > -40.0 && !(fabs(cur[i] - ref[i]) <= 0.01)) {
                        st = 1;
                        break;
                    }
            }
            note(t, ms, st);
            // keep a change only when it is clearly faster than the current setting timed beside it
            if (st == SBR_OK && ms < 0.99 * base_ms) {
                cur_ms = ms;
                bestt = t;
            } else if (st == SBR_OK) {
                cur_ms = std::min(cur_ms, base_ms);
            }
        }
    }
    c->tune = bestt;
    c->err.clear();
    if (n_trials) *n_trials = nt;
    if (best) *best = bestt;
    if (best_ms) *best_ms = cur_ms;
    return SBR_OK;
}

int sbr_get_hits(sbr_ctx* c, int64_t angle, int32_t* tri_ids, float* t, int32_t* n_bounce)
{
    if (!c) return SBR_ERR_ARG;
    if (!c->has_trace || !(c->trace_flags & SBR_TRACE_RECORD_HITS))
        return fail(c, SBR_ERR_STATE, "sbr_get_hits: last trace did not record hits");
    if (angle < 0 || angle >= (int64_t)c->ang.size()) return fail(c, SBR_ERR_ARG, "sbr_get_hits: angle out of range");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    const AngleHost& h = c->ang[(size_t)angle];
    const size_t np = (size_t)tiled_rays(h.grid, h.tw), B = (size_t)c->max_bounces;
    std::vector<int> ht(np * B), hn(np);
    std::vector<float> htt(np * B);
    CK(cudaMemcpyAsync(ht.data(), c->hit_tri.as<int>() + (size_t)h.ray_begin * B, sizeof(int) * np * B,
                       cudaMemcpyDeviceToHost, c->stream),
       "copy hits");
    CK(cudaMemcpyAsync(htt.data(), c->hit_t.as<float>() + (size_t)h.ray_begin * B, sizeof(float) * np * B,
                       cudaMemcpyDeviceToHost, c->stream),
       "copy hits");
    CK(cudaMemcpyAsync(hn.data(), c->hit_nb.as<int>() + h.ray_begin, sizeof(int) * np, cudaMemcpyDeviceToHost,
                       c->stream),
       "copy hits");
    CK(cudaStreamSynchronize(c->stream), "hits sync");
    // processing layout (tiles of W x 32 / W) -> ray id j * nu + i
    const long long W = 1ll << h.tw, nbu = (h.grid.nu + W - 1) / W;
    for (size_t p = 0; p < np; ++p) {
        const long long blk = (long long)(p >> 5), l = (long long)(p & 31);
        const long long i = (blk % nbu) * W + (l & (W - 1)), j = (blk / nbu) * (32 / W) + (l >> h.tw);
        if (i >= h.grid.nu || j >= h.grid.nv) continue;
        const size_t id = (size_t)(j * h.grid.nu + i);
        for (size_t b = 0; b < B; ++b) {
            if (tri_ids) tri_ids[id * B + b] = ht[p * B + b];
            if (t) t[id * B + b] = htt[p * B + b];
        }
        if (n_bounce) n_bounce[id] = hn[p];
    }
    return SBR_OK;
}

int sbr_get_records(sbr_ctx* c, int64_t angle, int64_t cap, int64_t* ray_ids, float* coef, double* path,
                    int64_t* n_out)
{
    if (!c) return SBR_ERR_ARG;
    if (!c->has_trace) return fail(c, SBR_ERR_STATE, "sbr_get_records: no trace results");
    if (angle < 0 || angle >= (int64_t)c->ang.size()) return fail(c, SBR_ERR_ARG, "sbr_get_records: angle out of range");
    const AngleHost& h = c->ang[(size_t)angle];
    if (n_out) *n_out = h.rec_count;
    const long long n = std::min<long long>(cap, h.rec_count);
    if (n <= 0) return SBR_OK;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    std::vector<Record> r((size_t)n);
    CK(cudaMemcpyAsync(r.data(), c->rec.as<Record>() + h.rec_begin, sizeof(Record) * (size_t)n, cudaMemcpyDeviceToHost,
                       c->stream),
       "copy records");
    CK(cudaStreamSynchronize(c->stream), "records sync");
    for (long long i = 0; i < n; ++i) {
        if (ray_ids) ray_ids[i] = r[(size_t)i].ray;
        if (coef)
            for (int q = 0; q < 5; ++q) coef[5 * i + q] = r[(size_t)i].c[q];
        if (path) path[i] = (double)r[(size_t)i].l_hi + (double)r[(size_t)i].l_lo;
    }
    return SBR_OK;
}

}  // extern "C"
