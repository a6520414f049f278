/*
 * sbr.h -- C ABI of libsbr, a GB300 (sm_103a) implementation of the
 * trace-integrate hot path of shooting and bouncing rays (SBR) for monostatic
 * radar cross section, after "BVH-Accelerated Ray Tracing for High-Frequency
 * Electromagnetic Backscattering" (arXiv 2604.09243).
 *
 * Pipeline (Sec. 4 and Fig. 1 of the paper):
 *   sbr_load_mesh    triangulated PEC surface                        (Sec. 4.1)
 *   sbr_build_bvh    LBVH over the triangles, SAH leaf collapse      (Sec. 4, BVH)
 *   sbr_trace        orthographic ray grid per aspect (Eq. L1-L3), multi-bounce
 *                    closest-hit transport with specular reflection and PEC
 *                    field update (Algorithm 2), compaction of valid hits
 *   sbr_po_integrate physical-optics ray-tube sum over valid hits only
 *                    (Eq. po_sum; vector form from Eq. em5/em6) and
 *                    sigma = 4 pi |A|^2 in dBsm (Sec. 4, after Eq. po_sum)
 *
 * Conventions shared by every call:
 *   - Angles in degrees. r = (cos el cos az, cos el sin az, sin el) points to the
 *     radar; the incident direction is k_inc = -r. V = theta_hat =
 *     (sin el cos az, sin el sin az, -cos el), H = phi_hat = (-sin az, cos az, 0).
 *   - Polarisation order HH, VV, HV, VH: first letter receive, second transmit.
 *   - Every call returns an int status (SBR_OK = 0, negative on error) and never
 *     aborts or throws across the ABI; sbr_last_error() gives the message.
 *   - All device work of a context is ordered on the context's CUDA stream.
 *     Calls that return results to host memory synchronise that stream.
 *   - A context is not thread safe: use one context per host thread.
 */
#ifndef SBR_H_
#define SBR_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SBR_VERSION_MAJOR 0
#define SBR_VERSION_MINOR 1

/* status codes */
#define SBR_OK 0
#define SBR_ERR_ARG (-1)            /* invalid argument (null pointer, size, index) */
#define SBR_ERR_CUDA (-2)           /* a CUDA runtime call failed */
#define SBR_ERR_OOM (-3)            /* device or pinned-host allocation failed */
#define SBR_ERR_STATE (-4)          /* call out of order (no mesh, no BVH, no trace) */
#define SBR_ERR_STACK_OVERFLOW (-5) /* a traversal needed more than the stack depth */
#define SBR_ERR_TIMEOUT (-6)        /* a bounded device wait gave up */
#define SBR_ERR_NODEV (-7)          /* no usable CUDA device */

/* polarisation mask bits for sbr_po_integrate */
#define SBR_POL_HH 1
#define SBR_POL_VV 2
#define SBR_POL_HV 4
#define SBR_POL_VH 8

/* po_mode for sbr_po_integrate: one form, optionally OR-ed with one phase precision */
#define SBR_PO_VECTOR 0           /* Stratton-Chu PO at the last hit (Eq. em5, em6) */
#define SBR_PO_PAPER_SCALAR 1     /* Eq. po_sum literally, Gamma = -1 (PEC) */
#define SBR_PHASE_COMPENSATED 0   /* k*L as a two-float product, reduced in cycles (default) */
#define SBR_PHASE_FP32 16         /* plain FP32 k*L and sincosf */
#define SBR_PHASE_FP64 32         /* FP64 k*L and sincos (slow on GB300) */

/* sbr_trace_opts.flags */
#define SBR_TRACE_PHASE_LITERAL_2R 1 /* scalar form uses e^{-j 2 k R}, R the summed path (Eq. po_sum as printed) */
#define SBR_TRACE_REQUIRE_ESCAPE 2   /* a ray still hitting after max_bounces is invalid (Sec. 4 text) */
#define SBR_TRACE_RECORD_HITS 4      /* keep per-ray, per-bounce hits for sbr_get_hits */
#define SBR_TRACE_COUNT_VISITS 8     /* count node visits and triangle tests into the stats */
#define SBR_TRACE_TIME_PASSES 16     /* time each transport pass with CUDA events into the stats */
#define SBR_TRACE_NO_GRAPH 32        /* sbr_submit_batch: enqueue the kernels directly, no CUDA graph */

typedef struct sbr_ctx sbr_ctx; /* opaque; owns the device copies of mesh, BVH and ray buffers */

/* BVH build options (Sec. 4: SAH cost C_T + SA(L)/SA(P) N_L C_I + SA(R)/SA(P) N_R C_I). */
typedef struct {
    int leaf_max;         /* largest leaf after the SAH collapse, 1..16 (default 4) */
    float cost_traverse;  /* C_T (default 1) */
    float cost_intersect; /* C_I (default 1) */
    int builder;          /* SBR_BVH_PLOC (0, default) or SBR_BVH_LBVH */
    int ploc_radius;      /* PLOC search radius in Morton order, 1..64 (0 = 16) */
} sbr_bvh_opts;
#define SBR_BVH_PLOC 0 /* agglomerative clustering of mutual nearest neighbours in the Morton order, close
                          to a full SAH tree (one host synchronisation per four clustering rounds) */
#define SBR_BVH_LBVH 1 /* Karras hierarchy over the Morton order, bottom-up refit */

/* Ray-grid and transport options of sbr_trace. A zeroed struct gives the defaults. */
typedef struct {
    double window_m; /* > 0: fixed square aperture of this side replaces Eq. L2 (N = ceil(W/ds)) */
    double offset_u; /* sub-cell shift of the whole grid along u, in units of the spacing */
    double offset_v; /* same along v */
    int flags;       /* SBR_TRACE_* */
    int chunk_rays;  /* rays per internal batch of aspects (0 = 2^27); bounds the live-ray queue
                        memory at 192 bytes per ray (292 with the ray pool, and its grouping, of a
                        trace of several chunks); an aspect larger than this is refused */
} sbr_trace_opts;

/* Counters of the last sbr_trace (summed over its angles). */
typedef struct {
    int64_t n_angles;
    int64_t rays_launched; /* sum of Nu*Nv (Eq. L3) */
    int64_t ray_bounces;   /* closest-hit queries on live rays, hit or miss */
    int64_t valid_rays;    /* rays with at least one hit (Algorithm 2 'valid') */
    int64_t node_visits;   /* only with SBR_TRACE_COUNT_VISITS */
    int64_t tri_tests;     /* only with SBR_TRACE_COUNT_VISITS */
    int64_t stack_overflows;
    int64_t kernel_launches; /* CUDA kernels this call enqueued */
    int64_t pass_launches;   /* transport-pass kernels among them (primary and bounce passes) */
    double pass_ms;          /* with SBR_TRACE_TIME_PASSES: summed device time of those passes */
    int64_t raster_tests;    /* only with SBR_TRACE_COUNT_VISITS: triangle tests of the rasterised primary hits
                                (included in tri_tests) */
    double primary_ms;       /* with SBR_TRACE_TIME_PASSES: the part of pass_ms spent in primary passes
                                (rasterisation included) */
    int64_t bounce_hits;     /* only with SBR_TRACE_COUNT_VISITS: hits processed by the bounce passes (reflection,
                                field update and candidate coefficients each) */
    int64_t listed_hits;     /* only with SBR_TRACE_COUNT_VISITS: rasterised primary hits whose state bounce pass 1
                                rebuilt from the hit list (their per-hit arithmetic runs there) */
    int64_t open_tests;      /* only with SBR_TRACE_COUNT_VISITS: triangle tests whose FP32 filter left the decision
                                open (taken again near the triangle, then in FP64 if still open) */
    int64_t fp64_tests;      /* only with SBR_TRACE_COUNT_VISITS: of those, the tests decided in FP64 */
    int64_t warp_node_visits; /* only with SBR_TRACE_COUNT_VISITS: over the bounce passes' warp-wide queries, 32 x the
                                 largest node visit count among the warp's lanes (node_visits of the bounce passes
                                 divided by it is the lane occupancy their traversal lengths allow) */
} sbr_trace_stats;

/* Per-aspect ray grid (Eq. L1-L3) exactly as sbr_trace generates it. */
typedef struct {
    int64_t nu, nv;          /* Eq. L3 */
    double lu, lv;           /* projected extents, Eq. L1 */
    double spacing;          /* ds (m); tube area dA = ds^2 */
    double eps;              /* origin offset after a hit: 1e-5 * bbox diagonal (m) */
    double rhat[3], khat[3]; /* direction to the radar and incident direction */
    double vhat[3], hhat[3]; /* V = theta_hat (aperture v), H = phi_hat (aperture u) */
    float p0[3];             /* origin of ray (0, 0), FP32 */
    float du[3], dv[3];      /* grid steps ds*u and ds*v, FP32 */
    float dir[3];            /* ray direction k_inc, FP32 */
} sbr_ray_grid;

/* Library version as major*100 + minor. */
int sbr_version(void);

/* Create a context on CUDA device `device`. `cuda_stream` is a cudaStream_t to
 * order all work on (e.g. torch.cuda.current_stream().cuda_stream), or NULL for
 * a stream the context creates and owns. The caller keeps ownership of a
 * stream it passes and must keep it alive until sbr_destroy. On failure *out is
 * NULL and the status is SBR_ERR_NODEV, SBR_ERR_CUDA or SBR_ERR_ARG. */
int sbr_create(sbr_ctx** out, int device, void* cuda_stream);

/* Free every device buffer of the context (after synchronising its stream). NULL is a no-op. */
void sbr_destroy(sbr_ctx* ctx);

/* Message of the last failed call on `ctx` (owned by the context, valid until the
 * next call on it); for ctx == NULL, the message of the last failed sbr_create
 * or sbr_po_integrate_noalloc. */
const char* sbr_last_error(const sbr_ctx* ctx);

/* Load a triangulated PEC surface (Sec. 4.1 of the paper; meshes come from the
 * caller, no file I/O). xyz: float32 [n_vert][3] metres; tri: int32 [n_tri][3]
 * vertex indices. on_device = 0: host pointers; 1: device pointers on the
 * context's device. The data are copied; the caller keeps ownership. Indices
 * outside [0, n_vert) and non-finite vertex coordinates give SBR_ERR_ARG. A
 * degenerate triangle, |e1 x e2|^2 <= 2^-40 |e1|^2 |e2|^2 in FP32 (repeated or
 * collinear vertices, slivers whose edge angle has a sine of at most 2^-20),
 * stays in the mesh but takes no hits. Replaces any previous mesh and drops
 * the trace results; it also computes the scene box and builds a BVH with the
 * default options (sbr_build_bvh rebuilds it with others). Synchronises. */
int sbr_load_mesh(sbr_ctx* ctx, const float* xyz, int64_t n_vert, const int32_t* tri, int64_t n_tri,
                  int on_device);

/* Scene bounding box [xmin, ymin, zmin, xmax, ymax, zmax] of the loaded mesh
 * (exact FP32 min/max of the vertices), written to host memory. */
int sbr_get_bbox(sbr_ctx* ctx, float* bbox6);

/* Build the BVH (Sec. 4, BVH paragraph; Algorithm 1 is the paper's host
 * builder, this is a GPU LBVH): 63-bit Morton codes of the triangle centroids,
 * device radix sort, Karras hierarchy, bottom-up AABB refit and SAH leaf
 * collapse with C_T, C_I and leaf_max from `opt` (NULL = defaults), triangles
 * reordered so each leaf is a contiguous range; then the 4-wide collapse of
 * that tree (sbr_tuning.bvh_width picks the one traversed). By default
 * (SBR_BVH_PLOC; also what sbr_load_mesh builds) the hierarchy comes from
 * nearest-neighbour clustering of the Morton-ordered triangles instead of the
 * Karras split (SBR_BVH_LBVH); leaf collapse and layout are the same.
 * Synchronises. The nodes reachable from the root are then renumbered in
 * depth-first order (the larger child first), so that each subtree is one
 * contiguous range of the node array; boxes, leaves and hits do not change. */
int sbr_build_bvh(sbr_ctx* ctx, const sbr_bvh_opts* opt);

/* Size of the current tree: triangles, binary nodes reachable from the root
 * (64 bytes each; the node array holds no others once built), nodes of its
 * 4-wide collapse (128 bytes each). SBR_ERR_STATE without a mesh. */
typedef struct {
    int64_t n_tri;
    int64_t n_nodes;
    int64_t n_nodes4;
} sbr_bvh_info;
int sbr_get_bvh_info(sbr_ctx* ctx, sbr_bvh_info* out);

/* Ray grid of one aspect for the loaded mesh (Eq. L1-L3), computed on the host.
 * ray_spacing_m = ds, margin_eta = eta of Eq. L2 (ignored when opt->window_m > 0).
 * Needs a loaded mesh but no device work. */
int sbr_ray_grid_for(sbr_ctx* ctx, double az_deg, double el_deg, double ray_spacing_m, double margin_eta,
                     const sbr_trace_opts* opt, sbr_ray_grid* out);

/* Same as sbr_ray_grid_for for an explicit scene box bbox6 (host, float[6] =
 * xmin, ymin, zmin, xmax, ymax, zmax); needs no context and no GPU. Ray (i, j)
 * of the grid starts at (p0 + i*du) + j*dv, each operation an FP32
 * round-to-nearest multiply or add (no fused multiply-add), and travels along dir. */
int sbr_ray_grid_box(const float* bbox6, double az_deg, double el_deg, double ray_spacing_m, double margin_eta,
                 const sbr_trace_opts* opt, sbr_ray_grid* out);

/* Trace every aspect of az_el_deg (host, [n_angles][2] = (az, el) degrees):
 * orthographic ray grid per aspect (Eq. L1-L3), up to max_bounces closest-hit
 * queries per ray with specular reflection d - 2 (d.n) n, PEC field update
 * E' = 2 (n.E) n - E and origin offset eps along the normal (Algorithm 2),
 * then compaction of the valid rays into a dense record buffer (Sec. 4,
 * trace-integrate decomposition). The records stay in the context until the
 * next sbr_trace or sbr_load_mesh; sbr_po_integrate reads them for any list of
 * frequencies. `opt` may be NULL; `stats` may be NULL (it is filled on return
 * and then the stream is synchronised). max_bounces in 1..128. The aspects
 * are traced in chunks of at most opt->chunk_rays rays; when there are several,
 * the bounces after the first run once over the rays of all chunks (a ray pool
 * the size of a chunk queue), which changes no ray's hits or records. */
int sbr_trace(sbr_ctx* ctx, const double* az_el_deg, int64_t n_angles, double ray_spacing_m, double margin_eta,
              int max_bounces, const sbr_trace_opts* opt, sbr_trace_stats* stats);

/* Bistatic variant of sbr_trace (the paper notes that monostatic SBR needs no
 * visibility function, Sec. 3 footnote; a bistatic one does): aspect a is lit
 * from az_el_tx[a] (the ray grid, as in sbr_trace) and observed from the
 * receiver direction az_el_rx[a] (host double [n][2], degrees, same axis
 * convention). The PO terms of the records radiate toward the receiver and are
 * projected on its H, V basis (pq = receive p, transmit q), the path becomes
 * L = k.o0 + sum t - r_rx.x_last, and a ray's last hit counts only if it sees
 * the receiver: the receiver lies on the side of the hit's oriented normal and
 * a query from the offset hit point toward the receiver meets no triangle
 * (its records are zero otherwise). Each visibility query counts as a
 * ray-bounce. sbr_po_integrate then gives the bistatic field (vector form; the
 * paper scalar form stays monostatic). With az_el_rx = az_el_tx the fields
 * equal the monostatic ones for rays whose last hit sees the radar. */
int sbr_trace_bistatic(sbr_ctx* ctx, const double* az_el_tx, const double* az_el_rx, int64_t n_angles,
                       double ray_spacing_m, double margin_eta, int max_bounces, const sbr_trace_opts* opt,
                       sbr_trace_stats* stats);

/* Physical-optics ray-tube sum over the valid hits of the last sbr_trace, for
 * every traced aspect and every frequency of freq_hz (host, n_freq values):
 *   E_pq = (-j k / 4 pi) sum_i c_pq,i e^{-j k L_i},  k = 2 pi f / c0,
 * with c_pq,i the tube's coefficient for receive p / transmit q (Eq. em6 in
 * SBR_PO_VECTOR; Eq. po_sum with Gamma = -1 in SBR_PO_PAPER_SCALAR, where
 * HH = VV = A and HV = VH = 0), then sigma = 4 pi |E|^2 and dBsm = 10 log10 sigma.
 * The partial sums are FP32 per block of tubes and FP64 across blocks, in a
 * fixed order (results are bitwise reproducible). pol_mask selects the
 * polarisations (SBR_POL_*); n_pol = popcount(pol_mask) outputs in the order
 * HH, VV, HV, VH. Outputs: E_re_im [n_angles][n_freq][n_pol][2] FP64 and
 * rcs_dbsm [n_angles][n_freq][n_pol] FP64 (either may be NULL), in host memory
 * (out_on_device = 0, synchronises) or device memory (1, stream ordered).
 * With one frequency (two with at most two polarisations) the records stream
 * through shared memory by bulk copies with bounded waits; a wait that gives up
 * makes the affected sums NaN and, with host outputs, returns SBR_ERR_TIMEOUT.
 * The sums are the same bit for bit either way. */
int sbr_po_integrate(sbr_ctx* ctx, const double* freq_hz, int64_t n_freq, int pol_mask, int po_mode,
                     double* E_re_im, double* rcs_dbsm, int out_on_device);

/* One request of a batch: an aspect with its own ray spacing and its own list
 * of frequencies (entries freq_offset .. freq_offset + n_freq - 1 of the
 * batch's frequency array). */
typedef struct {
    double az_deg, el_deg;
    double ray_spacing_m;  /* ds of this request (e.g. sbr_spacing_for(its highest frequency, rays/lambda)) */
    int64_t freq_offset;
    int32_t n_freq;
    int32_t reserved;
} sbr_request;

/* Batched trace-integrate (the paper's angular sweep, Sec. 4 last paragraph,
 * done inside one GPU): every request is traced once (Algorithm 2, Eq. L1-L3
 * with its own spacing) and its frequency-independent ray paths are integrated
 * for all of its frequencies (Eq. po_sum / em6), requests of uneven ray counts
 * packed into chunks of persistent-kernel passes. Consecutive chunks form
 * groups of at most four chunks' worth of records; the bounces after the first
 * run once over the rays of a group (the ray pool of sbr_trace), and a group is
 * integrated as soon as it is traced, so record memory stays bounded by a few
 * chunk sizes (opt->chunk_rays). Output row r0 + q (r0 = sum of n_freq over the earlier
 * requests) holds frequency q of a request: E_re_im [rows][n_pol][2],
 * rcs_dbsm [rows][n_pol], host (out_on_device = 0) or device (1) memory.
 * The call synchronises; it leaves no trace results behind (sbr_po_integrate
 * and sbr_get_records need sbr_trace). SBR_TRACE_RECORD_HITS is refused. */
int sbr_run_batch(sbr_ctx* ctx, const sbr_request* req, int64_t n_req, const double* freq_hz, int64_t n_freq_total,
                  double margin_eta, int max_bounces, int pol_mask, int po_mode, const sbr_trace_opts* opt,
                  double* E_re_im, double* rcs_dbsm, int out_on_device, sbr_trace_stats* stats);

/* Batched trace-integrate, asynchronous (same requests, frequency array,
 * options and output layout as sbr_run_batch, and the same results bit for
 * bit). The PO work lists are built on the device from the record counts, so
 * the whole batch runs with no host synchronisation: it is captured once as
 * one CUDA graph and launched on the ctx stream, and the call returns without
 * waiting. Submitting the same arguments again (requests, frequencies, eta,
 * bounces, polarisations, mode, options and output pointers) on the same mesh
 * replays the captured graph without planning again.
 *   E_dev, rcs_dev: DEVICE memory (either may be NULL) laid out as in
 *   sbr_run_batch; written when the ctx stream reaches the end of the graph.
 *   opt->flags: SBR_TRACE_REQUIRE_ESCAPE, SBR_TRACE_COUNT_VISITS as for
 *   sbr_trace; SBR_TRACE_NO_GRAPH enqueues the kernels directly each time;
 *   SBR_TRACE_RECORD_HITS and SBR_TRACE_TIME_PASSES are refused.
 * The plan owns its device buffers (ray queues for its largest chunk, record
 * and partial buffers sized for every ray being valid) until a submit with
 * other arguments or sbr_destroy; sbr_trace results are left untouched.
 * Errors found while planning are returned here; kernel-side conditions
 * (stack overflow) by sbr_sync. No counterpart in the paper: the paper's
 * sweep is a host loop over aspects. */
int sbr_submit_batch(sbr_ctx* ctx, const sbr_request* req, int64_t n_req, const double* freq_hz,
                     int64_t n_freq_total, double margin_eta, int max_bounces, int pol_mask, int po_mode,
                     const sbr_trace_opts* opt, double* E_dev, double* rcs_dev);
/* Wait for the last submitted batch and report its statistics as
 * sbr_run_batch does (kernel_launches: kernels per run of the batch).
 * SBR_ERR_STATE if nothing was submitted. */
int sbr_sync(sbr_ctx* ctx, sbr_trace_stats* stats);

/* ---- tuning ------------------------------------------------------------------
 * Launch and layout parameters of the trace-integrate path. None of them
 * changes any ray's hits or records; the ray tile and the PO item size change
 * the order of the FP32 partial sums, so fields agree to rounding across
 * settings and bit for bit between runs with the same setting. */
typedef struct {
    int tile_w;          /* rays of a warp form a tile_w x (32 / tile_w) patch; 1, 2, 4, 8, 16, 32 (default 8) */
    int blocks_per_sm;   /* resident 256-thread transport blocks per SM, 1..4 (default: occupancy limit) */
    int stack_depth;     /* traversal stack entries: 32, 64 or 128 (default 64); a query that needs more is
                            reported as a stack overflow (SBR_ERR_STACK_OVERFLOW) */
    int chunk_rays_log2; /* rays per chunk when opt->chunk_rays is 0: 2^20 .. 2^29 (default 27); a chunk's
                            two live-ray queues take 192 bytes per ray (about 100 GB at 2^29), and
                            sbr_trace over several chunks adds a ray pool of one queue's size */
    int po_item;         /* records per PO block: 512, 1024 or 2048 (default 1024) */
    int bvh_width;       /* 2: binary LBVH; 4: its 4-wide collapse (same boxes, fewer dependent fetches);
                            default 2 */
    int packet;          /* 1: the 32 rays of a warp walk the binary tree together (one broadcast fetch
                            per node, no divergence; each ray still tests only the boxes it enters);
                            needs bvh_width 2 and stack_depth <= 64; default 0 */
    int octant;          /* 1: traverse copies of the binary nodes stored per direction octant with the near
                            and far slab of each axis chosen in advance (no per-axis min/max; 8 x the node
                            memory, built on first use); needs bvh_width 2 and packet 0; default 0 */
    int silhouette;      /* 1: before the primary pass, rasterise every triangle's widened projection onto
                            the ray grid and skip the query of rays outside all of them (sure misses: no
                            hit, not counted as ray-bounces); default 0 */
    int raster;          /* 1: find the primary hits by rasterisation instead of traversal: every triangle
                            runs the FP32 test for each grid ray of its widened projected box and a 64-bit
                            atomic minimum of (t, original index) keeps the closest hit, so the hits are
                            those of the traversal; an aspect with a triangle spanning more than 2^14 grid
                            cells traverses instead. The silhouette mask is then not used. Default 1 */
} sbr_tuning;
int sbr_get_tuning(const sbr_ctx* ctx, sbr_tuning* out);
/* SBR_ERR_ARG for a value outside the ranges above. */
int sbr_set_tuning(sbr_ctx* ctx, const sbr_tuning* t);

/* One configuration tried by sbr_autotune: its fastest time per run of the
 * sample batch (host wall clock of sbr_run_batch) and status: 0 accepted,
 * 1 refused because its dBsm differ from the starting configuration's by more
 * than 0.01 dB where those are above -40 dBsm, < 0 the error code of the run
 * (e.g. SBR_ERR_STACK_OVERFLOW for a stack too shallow for the mesh). */
typedef struct {
    sbr_tuning tuning;
    double ms;
    int status;
    int reserved;
} sbr_tune_trial;

/* Autotuner: times sbr_run_batch on the given sample batch (arguments as for
 * sbr_run_batch) under the current setting and then, one parameter at a
 * time (traversal: binary / 4-wide / warp-cooperative / octant copies, blocks per SM, ray
 * tile, stack depth, PO item, chunk size, silhouette mask, rasterised primary hits), under
 * each alternative value, keeping a change when it is more than 1 % faster and its results
 * agree (see sbr_tune_trial). Each timing is the fastest of `reps` runs after one
 * warm-up run; a candidate's runs alternate with runs of the current setting,
 * and the two are compared on those. Leaves the fastest accepted setting on the
 * ctx and returns it in *best, and in *best_ms the fastest time measured for it
 * (its own trial or a run beside a later candidate). trials: host array of
 * capacity trial_cap (may be NULL); *n_trials receives the number of settings
 * tried. Synchronises; takes 1 + 2 reps runs of the sample per setting tried. */
int sbr_autotune(sbr_ctx* ctx, const sbr_request* req, int64_t n_req, const double* freq_hz, int64_t n_freq_total,
                 double margin_eta, int max_bounces, int pol_mask, int po_mode, const sbr_trace_opts* opt, int reps,
                 sbr_tune_trial* trials, int trial_cap, int* n_trials, sbr_tuning* best, double* best_ms);

/* Per-ray hits of traced aspect `angle` (needs SBR_TRACE_RECORD_HITS), for
 * parity checks; ray id = j * nu + i. Host outputs (any may be NULL):
 * tri_ids [nu*nv][max_bounces] original triangle index or -1, t [nu*nv][max_bounces]
 * hit distance along each leg, n_bounce [nu*nv]. Synchronises. */
int sbr_get_hits(sbr_ctx* ctx, int64_t angle, int32_t* tri_ids, float* t, int32_t* n_bounce);

/* Dense valid-hit records of traced aspect `angle`, in ray order, for parity
 * checks. Host outputs of capacity `cap` records (any may be NULL):
 * ray_ids (j*nu + i), coef [.][5] = (HH, VV, HV, VH, scalar) tube coefficients,
 * path [.] = L in metres. *n_out receives the record count. Synchronises. */
int sbr_get_records(sbr_ctx* ctx, int64_t angle, int64_t cap, int64_t* ray_ids, float* coef, double* path,
                    int64_t* n_out);

/* ---- learned surrogate ------------------------------------------------------
 * A Fourier-feature MLP that learns the complex HH/VV field from SBR samples
 * (its training data come from sbr_trace/sbr_po_integrate or sbr_run_batch):
 * inputs (az, el, f) -> (sin az, cos az, el / 30 deg, log f mapped from
 * [1, 12] GHz to [-1, 1]) -> n_fourier features [sin 2 pi B x, cos 2 pi B x],
 * B ~ N(0, fourier_sigma^2) -> depth GELU layers of `width` -> 4 outputs
 * (Re HH, Im HH, Re VV, Im VV). Hidden layers run in BF16 with FP32
 * accumulation on the tcgen05 tensor-core GEMM (forward and backward); FP32
 * master weights, Adam, mean-squared error on targets divided by their RMS.
 * n_members independently initialised networks form an ensemble; the spread
 * of their |E|^2 in dB marks points where the caller should fall back to SBR. */
typedef struct sbr_surrogate sbr_surrogate;
typedef struct {
    int n_members;       /* ensemble size (default 4) */
    int width;           /* hidden width, a multiple of 128 (default 512) */
    int depth;           /* hidden GELU layers, 1..16 (default 6) */
    int n_fourier;       /* Fourier features, a multiple of 128 (default 256) */
    float fourier_sigma; /* standard deviation of the Fourier matrix (default 4) */
    uint64_t seed;       /* initialisation and shuffling seed (default 1) */
} sbr_surrogate_opts;

/* Create on CUDA device `device`, work ordered on cuda_stream (NULL: own stream); opt NULL = defaults. */
int sbr_surrogate_create(sbr_surrogate** out, int device, void* cuda_stream, const sbr_surrogate_opts* opt);
void sbr_surrogate_destroy(sbr_surrogate* s);
const char* sbr_surrogate_last_error(const sbr_surrogate* s);
/* Parameters per member: [W_0 (width x n_fourier), b_0, W_1 (width x width), b_1, ..., W_head (4 x width),
 * b_head (4)], FP32, row-major [out][in]. */
int64_t sbr_surrogate_num_params(const sbr_surrogate* s);
/* Copy member `member`'s parameters out to host `get` and/or in from host `set` (either may be NULL). */
int sbr_surrogate_params(sbr_surrogate* s, int member, float* get, const float* set);
/* Member `member`'s Fourier matrix B, host float [n_fourier / 2][4]. */
int sbr_surrogate_fourier(sbr_surrogate* s, int member, float* B);
/* Train every member for `epochs` epochs of shuffled mini-batches of `batch` samples (a multiple of 128;
 * an incomplete last batch of an epoch is dropped). x: host double [n][3] = (az deg, el deg, f Hz);
 * y: host double [n][4] = (Re HH, Im HH, Re VV, Im VV). loss_per_epoch: host float [n_members][epochs]
 * (mean squared error of the scaled targets) or NULL. Adam (0.9, 0.999); the learning rate follows a
 * cosine schedule from `lr` down to lr / 100 over the call's steps. Synchronises. */
int sbr_surrogate_train(sbr_surrogate* s, const double* x, const double* y, int64_t n, int epochs, int batch,
                        float lr, float* loss_per_epoch);
/* Loss and parameter gradients of member `member` on one batch (n a multiple of 128), parameters unchanged;
 * for gradient checks. grads: host float [num_params] in the parameter layout. Targets are divided by
 * the scale of the last sbr_surrogate_train (1 before any training). */
int sbr_surrogate_grads(sbr_surrogate* s, int member, const double* x, const double* y, int64_t n, double* loss,
                        float* grads);
/* Ensemble prediction at n points x (host double [n][3]): y_mean host double [n][4] (mean over members, in
 * the units of the training targets) and spread_db host float [n] (over HH and VV, the largest range across
 * members of 10 log10 |E|^2). Either output may be NULL. Synchronises. */
int sbr_surrogate_predict(sbr_surrogate* s, const double* x, int64_t n, double* y_mean, float* spread_db);

/* The tensor-core GEMM the surrogate runs on (tcgen05, TMA, FP32 accumulation in tensor memory):
 * C [M x N] (FP32, device, row stride ldc) = A [M x K] B^T, A and B BF16 on the device with K contiguous
 * (row strides lda, ldb, multiples of 8). M and N multiples of 128, K a multiple of 64. Synchronises
 * the stream; SBR_ERR_TIMEOUT if a bounded wait inside the kernel gave up. */
int sbr_gemm_bf16_tn(const void* A, int lda, const void* B, int ldb, int M, int N, int K, float* C, int ldc,
                     void* cuda_stream);
/* The same GEMM, only enqueued on the stream (no synchronisation): for callers that launch many and time them
 * on the device. err_dev: a device int the caller zeroes beforehand; a kernel whose bounded wait gave up sets
 * it to 1 (the caller reads it after synchronising). Returns SBR_ERR_ARG for a bad shape or pointer and
 * SBR_ERR_CUDA if the launch failed. */
int sbr_gemm_bf16_tn_async(const void* A, int lda, const void* B, int ldb, int M, int N, int K, float* C, int ldc,
                           int* err_dev, void* cuda_stream);

/* ---- allocation-free PO sum ------------------------------------------------
 * The paper has no counterpart of this call; it exists for callers that cannot
 * allocate device memory where they need the sum: plug-ins running inside an
 * application that owns and budgets all device memory, loops that must not
 * enter the allocator (whose calls can synchronise the device). It computes
 * what sbr_po_integrate computes, with the same kernels,
 * from caller-provided device records, and keeps all scratch in one fixed
 * file-scope device array (about 9 MB, held by every GPU that loads the
 * library until the process exits). It calls no cudaMalloc/cudaFree.
 *
 *   records      device, n_records x 32 bytes, each record 8 x 32-bit words:
 *                float c[5] (HH, VV, HV, VH, scalar-form coefficient), float L_hi,
 *                float L_lo (path L = L_hi + L_lo in metres), int ray id (unused);
 *                the layout sbr_trace produces (see sbr_get_records for values)
 *   rec_offsets  host, [n_angles + 1]: records of aspect a are
 *                [rec_offsets[a], rec_offsets[a + 1]); rec_offsets[0] = 0
 *   freq_hz      host, n_freq frequencies > 0
 *   pol_mask, po_mode  as for sbr_po_integrate
 *   E_re_im, rcs_dbsm  device outputs laid out as for sbr_po_integrate (one may be NULL)
 *   cuda_stream  stream to order the work on (NULL = legacy default stream)
 * Limits: n_angles <= SBR_NOALLOC_MAX_ANGLES, n_freq <= SBR_NOALLOC_MAX_FREQ,
 * at most SBR_NOALLOC_MAX_ITEMS blocks of 1024 records in total, and
 * blocks x n_freq x n_pol x 16 bytes <= SBR_NOALLOC_PARTIAL_BYTES; larger
 * requests return SBR_ERR_ARG with the reason in sbr_last_error(NULL).
 * The first call on a device looks up the array's device address (make that
 * first call before any stream capture). Every call reuses the same array and
 * overwrites what it reads, so calls that overlap on the GPU (other streams,
 * other host threads) race: order them. The small tables are copied from
 * pageable host memory under one lock: the call returns once the work is
 * enqueued and its tables are read, which can mean waiting for work already
 * queued on cuda_stream, and calls from several host threads take turns. */
#define SBR_NOALLOC_MAX_ANGLES 4096
#define SBR_NOALLOC_MAX_FREQ 256
#define SBR_NOALLOC_MAX_ITEMS 16384
#define SBR_NOALLOC_PARTIAL_BYTES (8u << 20)
int sbr_po_integrate_noalloc(const void* records, const int64_t* rec_offsets, int64_t n_angles, const double* freq_hz,
                             int64_t n_freq, int pol_mask, int po_mode, double* E_re_im, double* rcs_dbsm,
                             void* cuda_stream);

/* Measured peaks for the traversal's roofline (no counterpart in the paper; its
 * roofline needs the L2 bandwidth, which bounds the tree and triangle fetches
 * while they fit in L2, and the FP32 rate of the intersection arithmetic).
 *
 * sbr_probe_l2_bandwidth: reads a device buffer of `bytes` (>= 1 MiB; pick a
 * size below the L2 capacity) `passes` times (1..1000) with loads that bypass
 * L1, after one warm-up read, and writes the read rate in GB/s (1e9 bytes/s)
 * to *gb_per_s (host). sbr_probe_fp32_fma: eight independent FP32 fused
 * multiply-add chains on every thread of 8 blocks of 256 per SM; writes
 * TFLOP/s (two operations per fused multiply-add) to *tflops (host).
 * Both run on a stream of their own on `device`, time one launch with CUDA
 * events, allocate and free their buffers themselves, and return SBR_OK,
 * SBR_ERR_ARG, SBR_ERR_OOM or SBR_ERR_CUDA. */
int sbr_probe_l2_bandwidth(int device, int64_t bytes, int passes, double* gb_per_s);
int sbr_probe_fp32_fma(int device, double* tflops);

/* Ray spacing for `rays_per_lambda` rays per wavelength at frequency f_max_hz:
 * ds = c0 / (f_max_hz * rays_per_lambda); the paper's sampling rule (Sec. 4)
 * asks for ds <= lambda / 5. Returns a negative value for bad arguments. */
double sbr_spacing_for(double f_max_hz, double rays_per_lambda);

#ifdef __cplusplus
}
#endif

#endif /* SBR_H_ */
