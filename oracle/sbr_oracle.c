/*
 * sbr_oracle.c -- plain, slow, FP64 CPU oracle of the SBR trace-integrate path
 * of "BVH-Accelerated Ray Tracing for High-Frequency Electromagnetic
 * Backscattering" (arXiv 2604.09243).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library calls, links or
 * loads this file. It is used by the tests, by the smoke check and by the CPU
 * baseline leg of the benchmark. It shares no code, header, table or constant
 * generator with the CUDA path; both follow the same written conventions
 * (listed below), each in its own code.
 *
 * What it computes, step by step in the paper's order:
 *   1. Ray grid on the aperture plane (Sec. 4, Eq. L1-L3).
 *   2. Closest hit: brute force over every triangle, or the paper's median-split
 *      BVH (Algorithm 1) with a stack traversal, near child first (Sec. 4).
 *   3. Multi-bounce transport (Algorithm 2): x = o + t d, R += t, N += 1,
 *      specular reflection d - 2(d.n)n, new origin offset by eps along n.
 *   4. Physical-optics ray-tube sum over valid rays (Eq. po_sum; vector form
 *      from Eq. em5 / em6) and sigma = 4 pi |A|^2 (Sec. 4).
 *   5. Mie series of a PEC sphere (textbook Riccati-Bessel form), the check
 *      the paper validates against (Sec. 5.1).
 *
 * Readings of points the paper leaves open (each also taken by the GPU path):
 *   - Axes: r = (cos el cos az, cos el sin az, sin el) points to the radar,
 *     k_inc = -r, V = theta_hat = (sin el cos az, sin el sin az, -cos el),
 *     H = phi_hat = (-sin az, cos az, 0); aperture basis u = H, v = V.
 *   - Aperture: N = ceil(x - 1e-9) for x = (1+eta) L / ds (Eq. L3) or, with a
 *     fixed square window W, x = W / ds. Grid origin
 *       P0 = c - D k + (0.5 - Nu/2 + du) ds u + (0.5 - Nv/2 + dv) ds v,
 *     c = bbox centre, D = diag/2 + 1 m, (du, dv) an optional sub-cell offset;
 *     P0, ds*u, ds*v and k are rounded once to FP32 and ray (i, j) starts at
 *     o = (P0 + i*U) + j*V evaluated in FP32 without fused multiply-add, so both
 *     sides trace bit-identical rays; the oracle then continues in FP64.
 *   - Intersection: the exact test of the ray o + t d against the closed
 *     triangle (inclusive edges, t > 0) in Moller-Trumbore form, evaluated in
 *     FP64 on the FP32 ray and the FP32 vertices (edge differences, products
 *     and the decision carry rounding errors near 1e-16 relative, far inside the
 *     1e-6 edge band). The triangle just left is skipped, and the closest hit is
 *     the smallest (t, original triangle index) pair.
 *   - Ray state. The paper traces in FP32, so each bounce's ray is stored in
 *     FP32: every stored value is the FP32 rounding of its defining formula,
 *     evaluated on the previous FP32 state (the primary rays follow the grid
 *     rule above):
 *       n32 = fl32(N / |N|), N = (v1 - v0) x (v2 - v0)     (FP64, per triangle)
 *       t32 = fl32(((v0 - o) . n32) / (d . n32))   (hit distance to the plane of
 *             n32 through v0; the hit triangle itself is decided exactly)
 *       x   = fl32(o + t32 d),  c = fl32(d . n32)
 *       d'  = fl32(d - 2 c n32),  o' = fl32(x + eps32 nf),
 *     with nf = n32 turned toward the incoming side (sign of d . n32) and
 *     eps32 = fl32(1e-5 * bbox diagonal). Paths, fields and PO sums stay FP64.
 *   - Degenerate triangle (no hits): |N|^2 <= (2^-20 |e1|^2)(2^-20 |e2|^2) in
 *     FP64 (sine of the edge angle at most 2^-20).
 *   - Path L = k.o0 + sum t_b + k.x_last (monostatic round trip to a reference
 *     plane through the world origin); for one bounce this is 2 k.x1, i.e. the
 *     paper's e^{-j2kR} up to a constant phase. PHASE_LITERAL uses 2 (k.o0 + R).
 *   - Vector mode: at the last hit, J = 2 n x (d x E), dS = dA / |n.d|,
 *     contribution dS [J - (J.r) r] . p e^{-jkL}, prefactor -jk/(4 pi).
 *   - Scalar mode (Eq. po_sum literally, Gamma = -1): coefficient
 *     2 dA (n0 . -k_inc) (-1)^N with prefactor +jk/(4 pi); it is stored negated
 *     so both modes share the prefactor -jk/(4 pi).
 *   - Valid: N >= 1 (Algorithm 2); REQUIRE_ESCAPE also drops rays whose path is
 *     still hitting after B_max bounces.
 *   - Edge band: at some bounce the hit's smallest barycentric is < 1e-6, or a
 *     second candidate lies within 1e-6 (relative) of the closest t.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_C0 299792458.0
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ vectors */
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------ frame (Eq. L1-L3) */
typedef struct {
    double az_deg, el_deg;
    double rhat[3], khat[3], vhat[3], hhat[3];
    double centre[3], diag, D, Lu, Lv;
    double spacing, dA, eps;
    int64_t nu, nv;
    float P0[3], U[3], V[3], d[3];
    /* receiver (bistatic): direction to the receiver and its H, V basis; equal to
     * the transmitter's unless orc_frame_set_receiver was called */
    int bistatic;
    double rx_rhat[3], rx_hhat[3], rx_vhat[3];
    float rx_r32[3];
} orc_frame;

int orc_make_frame(const float* bbox, double az_deg, double el_deg, double spacing, double eta,
                   double window, double off_u, double off_v, orc_frame* f)
{
    if (!bbox || !f || !(spacing > 0.0)) return -1;
    memset(f, 0, sizeof(*f));
    f->az_deg = az_deg;
    f->el_deg = el_deg;
    double a = az_deg * (ORC_PI / 180.0), e = el_deg * (ORC_PI / 180.0);
    double ca = cos(a), sa = sin(a), ce = cos(e), se = sin(e);
    f->rhat[0] = ce * ca; f->rhat[1] = ce * sa; f->rhat[2] = se;
    for (int c = 0; c < 3; ++c) f->khat[c] = -f->rhat[c];
    f->vhat[0] = se * ca; f->vhat[1] = se * sa; f->vhat[2] = -ce;
    f->hhat[0] = -sa; f->hhat[1] = ca; f->hhat[2] = 0.0;
    double lo[3], hi[3], s2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        lo[c] = (double)bbox[c];
        hi[c] = (double)bbox[3 + c];
        f->centre[c] = 0.5 * (lo[c] + hi[c]);
        s2 += (hi[c] - lo[c]) * (hi[c] - lo[c]);
    }
    f->diag = sqrt(s2);
    f->D = 0.5 * f->diag + 1.0;
    /* Eq. L1: project the eight corners onto u and v */
    double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    for (int m = 0; m < 8; ++m) {
        double p[3] = {(m & 1) ? hi[0] : lo[0], (m & 2) ? hi[1] : lo[1], (m & 4) ? hi[2] : lo[2]};
        double pu = dot3(p, f->hhat), pv = dot3(p, f->vhat);
        if (pu < umin) umin = pu;
        if (pu > umax) umax = pu;
        if (pv < vmin) vmin = pv;
        if (pv > vmax) vmax = pv;
    }
    f->Lu = umax - umin;
    f->Lv = vmax - vmin;
    double xu, xv;
    if (window > 0.0) {
        xu = window / spacing;
        xv = xu;
    } else { /* Eq. L2, L3 */
        xu = (1.0 + eta) * f->Lu / spacing;
        xv = (1.0 + eta) * f->Lv / spacing;
    }
    f->nu = (int64_t)ceil(xu - 1e-9);
    f->nv = (int64_t)ceil(xv - 1e-9);
    if (f->nu < 1) f->nu = 1;
    if (f->nv < 1) f->nv = 1;
    f->spacing = spacing;
    f->dA = spacing * spacing;
    f->eps = 1e-5 * f->diag;
    double au = (0.5 - 0.5 * (double)f->nu + off_u) * spacing;
    double av = (0.5 - 0.5 * (double)f->nv + off_v) * spacing;
    for (int c = 0; c < 3; ++c) {
        f->P0[c] = (float)(((f->centre[c] - f->D * f->khat[c]) + au * f->hhat[c]) + av * f->vhat[c]);
        f->U[c] = (float)(spacing * f->hhat[c]);
        f->V[c] = (float)(spacing * f->vhat[c]);
        f->d[c] = (float)f->khat[c];
    }
    for (int c = 0; c < 3; ++c) {
        f->rx_rhat[c] = f->rhat[c];
        f->rx_hhat[c] = f->hhat[c];
        f->rx_vhat[c] = f->vhat[c];
        f->rx_r32[c] = (float)f->rhat[c];
    }
    f->bistatic = 0;
    return 0;
}

/* Bistatic receiver at (az, el): same axis convention as the transmitter. The
 * PO terms radiate toward it and are projected on its H, V basis; the last hit
 * of a ray contributes only if it sees the receiver (visibility test). */
int orc_frame_set_receiver(orc_frame* f, double az_deg, double el_deg)
{
    if (!f) return -1;
    double a = az_deg * (ORC_PI / 180.0), e = el_deg * (ORC_PI / 180.0);
    double ca = cos(a), sa = sin(a), ce = cos(e), se = sin(e);
    f->rx_rhat[0] = ce * ca; f->rx_rhat[1] = ce * sa; f->rx_rhat[2] = se;
    f->rx_vhat[0] = se * ca; f->rx_vhat[1] = se * sa; f->rx_vhat[2] = -ce;
    f->rx_hhat[0] = -sa; f->rx_hhat[1] = ca; f->rx_hhat[2] = 0.0;
    for (int c = 0; c < 3; ++c) f->rx_r32[c] = (float)f->rx_rhat[c];
    f->bistatic = 1;
    return 0;
}

/* FP32 ray of grid point (i, j); the build uses -ffp-contract=off */
void orc_ray(const orc_frame* f, int64_t i, int64_t j, float* o, float* d)
{
    float fi = (float)i, fj = (float)j;
    for (int c = 0; c < 3; ++c) {
        float a = fi * f->U[c];
        float b = f->P0[c] + a;
        float g = fj * f->V[c];
        o[c] = b + g;
        d[c] = f->d[c];
    }
}

/* ------------------------------------------------------------------ mesh + BVH (Algorithm 1) */
typedef struct {
    double lo[3], hi[3];
    int64_t left, right;  /* children (internal) */
    int64_t first, count; /* triangle range in `order` (leaf when count > 0) */
} orc_node;

typedef struct {
    int64_t nt;
    double* v0;  /* [nt][3] */
    double* e1;  /* [nt][3] v1 - v0 (exact: a difference of FP32 values) */
    double* e2;  /* [nt][3] v2 - v0 */
    float* n32;  /* [nt][3] FP32 rounding of the unit normal e1 x e2 / |e1 x e2| (0 when degenerate) */
    double* cen; /* [nt][3] centroid */
    double* tlo; /* [nt][3] triangle AABB, widened by a few FP64 rounding units */
    double* thi;
    unsigned char* deg; /* [nt] 1: degenerate, takes no hits */
    float bbox[6];
    orc_node* nodes;
    int64_t n_nodes, cap_nodes;
    int64_t* order;
    int leaf_size;
} orc_mesh;

void orc_mesh_free(orc_mesh* m)
{
    if (!m) return;
    free(m->v0); free(m->e1); free(m->e2); free(m->n32); free(m->cen); free(m->tlo); free(m->thi);
    free(m->deg);
    free(m->nodes); free(m->order);
    free(m);
}

/* Refuses bad indices and non-finite coordinates (NULL). A degenerate
 * triangle is kept but takes no hits: |e1 x e2|^2 <= (2^-20 |e1|^2)(2^-20 |e2|^2)
 * in FP64 (cross product, squared lengths and products in that order), so the
 * sine of the angle between its edges is at most 2^-20; repeated or collinear
 * vertices give zero. The paper assumes a valid surface mesh; such a triangle
 * has no usable normal to reflect about. */
orc_mesh* orc_mesh_create(const float* xyz, int64_t nv, const int32_t* tri, int64_t nt)
{
    if (!xyz || !tri || nt < 1 || nv < 3) return NULL;
    for (int64_t i = 0; i < 3 * nv; ++i)
        if (!isfinite(xyz[i])) return NULL;
    orc_mesh* m = (orc_mesh*)calloc(1, sizeof(orc_mesh));
    m->nt = nt;
    size_t b = sizeof(double) * 3 * (size_t)nt;
    m->v0 = malloc(b); m->e1 = malloc(b); m->e2 = malloc(b);
    m->cen = malloc(b); m->tlo = malloc(b); m->thi = malloc(b);
    m->n32 = malloc(sizeof(float) * 3 * (size_t)nt);
    m->deg = malloc((size_t)nt);
    for (int c = 0; c < 3; ++c) { m->bbox[c] = INFINITY; m->bbox[3 + c] = -INFINITY; }
    for (int64_t v = 0; v < nv; ++v)
        for (int c = 0; c < 3; ++c) {
            float x = xyz[3 * v + c];
            if (x < m->bbox[c]) m->bbox[c] = x;
            if (x > m->bbox[3 + c]) m->bbox[3 + c] = x;
        }
    for (int64_t k = 0; k < nt; ++k) {
        int32_t ia = tri[3 * k], ib = tri[3 * k + 1], ic = tri[3 * k + 2];
        if (ia < 0 || ib < 0 || ic < 0 || ia >= nv || ib >= nv || ic >= nv) { orc_mesh_free(m); return NULL; }
        double A[3], B[3], C[3];
        for (int c = 0; c < 3; ++c) {
            A[c] = xyz[3 * ia + c]; B[c] = xyz[3 * ib + c]; C[c] = xyz[3 * ic + c];
            m->v0[3 * k + c] = A[c];
            m->e1[3 * k + c] = B[c] - A[c];
            m->e2[3 * k + c] = C[c] - A[c];
            m->cen[3 * k + c] = (A[c] + B[c] + C[c]) / 3.0;
            m->tlo[3 * k + c] = fmin(A[c], fmin(B[c], C[c]));
            m->thi[3 * k + c] = fmax(A[c], fmax(B[c], C[c]));
        }
        /* the exact hit lies in the triangle's box; widen it by a few FP64
         * rounding units so the FP64 slab test cannot cull a flat (axis-aligned)
         * triangle's box on rounding */
        double ext = 0.0, mag = 0.0;
        for (int c = 0; c < 3; ++c) {
            ext = fmax(ext, m->thi[3 * k + c] - m->tlo[3 * k + c]);
            mag = fmax(mag, fmax(fabs(m->tlo[3 * k + c]), fabs(m->thi[3 * k + c])));
        }
        double grow = (ext + mag) * 0x1p-36 + 1e-30;
        for (int c = 0; c < 3; ++c) {
            m->tlo[3 * k + c] -= grow;
            m->thi[3 * k + c] += grow;
        }
        double n[3];
        cross3(m->e1 + 3 * k, m->e2 + 3 * k, n);
        const double nn = dot3(n, n), l1 = dot3(m->e1 + 3 * k, m->e1 + 3 * k), l2 = dot3(m->e2 + 3 * k, m->e2 + 3 * k);
        m->deg[k] = nn <= (l1 * 0x1p-20) * (l2 * 0x1p-20);
        const double ln = sqrt(nn);
        for (int c = 0; c < 3; ++c) m->n32[3 * k + c] = m->deg[k] ? 0.0f : (float)(n[c] / ln);
    }
    return m;
}

/* FP32 unit normals of the triangles [nt][3] (0 for a degenerate one) */
void orc_mesh_normals(const orc_mesh* m, float* out)
{
    memcpy(out, m->n32, sizeof(float) * 3 * (size_t)m->nt);
}

int64_t orc_mesh_n_degenerate(const orc_mesh* m)
{
    int64_t c = 0;
    for (int64_t k = 0; m && k < m->nt; ++k) c += m->deg[k];
    return c;
}

void orc_mesh_bbox(const orc_mesh* m, float* out)
{
    memcpy(out, m->bbox, sizeof(float) * 6);
}

static const orc_mesh* g_sort_mesh;
static int g_sort_axis;
static int cmp_centroid(const void* pa, const void* pb)
{
    int64_t a = *(const int64_t*)pa, b = *(const int64_t*)pb;
    double ca = g_sort_mesh->cen[3 * a + g_sort_axis], cb = g_sort_mesh->cen[3 * b + g_sort_axis];
    if (ca < cb) return -1;
    if (ca > cb) return 1;
    return (a < b) ? -1 : (a > b);
}

static int64_t bvh_build_rec(orc_mesh* m, int64_t first, int64_t count)
{
    if (m->n_nodes == m->cap_nodes) {
        m->cap_nodes = m->cap_nodes ? 2 * m->cap_nodes : 1024;
        m->nodes = (orc_node*)realloc(m->nodes, sizeof(orc_node) * (size_t)m->cap_nodes);
    }
    int64_t id = m->n_nodes++; /* allocated before the children: preorder */
    orc_node nd;
    for (int c = 0; c < 3; ++c) { nd.lo[c] = INFINITY; nd.hi[c] = -INFINITY; }
    for (int64_t i = first; i < first + count; ++i) {
        int64_t k = m->order[i];
        for (int c = 0; c < 3; ++c) {
            nd.lo[c] = fmin(nd.lo[c], m->tlo[3 * k + c]);
            nd.hi[c] = fmax(nd.hi[c], m->thi[3 * k + c]);
        }
    }
    nd.left = nd.right = -1;
    if (count <= m->leaf_size) {
        nd.first = first;
        nd.count = count;
        m->nodes[id] = nd;
        return id;
    }
    /* median split along the longest axis of the node AABB */
    int axis = 0;
    double ext[3] = {nd.hi[0] - nd.lo[0], nd.hi[1] - nd.lo[1], nd.hi[2] - nd.lo[2]};
    if (ext[1] > ext[axis]) axis = 1;
    if (ext[2] > ext[axis]) axis = 2;
    g_sort_mesh = m;
    g_sort_axis = axis;
    qsort(m->order + first, (size_t)count, sizeof(int64_t), cmp_centroid);
    int64_t nl = count / 2;
    nd.first = 0;
    nd.count = 0;
    m->nodes[id] = nd;
    int64_t l = bvh_build_rec(m, first, nl);
    int64_t r = bvh_build_rec(m, first + nl, count - nl);
    m->nodes[id].left = l;
    m->nodes[id].right = r;
    return id;
}

int orc_mesh_build_bvh(orc_mesh* m, int leaf_size)
{
    if (!m || leaf_size < 1) return -1;
    free(m->nodes);
    free(m->order);
    m->nodes = NULL;
    m->n_nodes = m->cap_nodes = 0;
    m->leaf_size = leaf_size;
    m->order = (int64_t*)malloc(sizeof(int64_t) * (size_t)m->nt);
    for (int64_t k = 0; k < m->nt; ++k) m->order[k] = k;
    bvh_build_rec(m, 0, m->nt);
    return 0;
}

int64_t orc_mesh_bvh_nodes(const orc_mesh* m) { return m ? m->n_nodes : 0; }

/* ------------------------------------------------------------------ intersection */
/* Moller-Trumbore in FP64 with inclusive edges; returns 1 on a hit with t > 0 */
static int tri_hit(const orc_mesh* m, int64_t k, const double* o, const double* d, double* t, double* bmin)
{
    const double *v0 = m->v0 + 3 * k, *e1 = m->e1 + 3 * k, *e2 = m->e2 + 3 * k;
    double p[3], q[3], s[3];
    if (m->deg[k]) return 0;
    cross3(d, e2, p);
    double det = dot3(e1, p);
    if (det == 0.0) return 0;
    for (int c = 0; c < 3; ++c) s[c] = o[c] - v0[c];
    double u = dot3(s, p) / det;
    if (u < 0.0 || u > 1.0) return 0;
    cross3(s, e1, q);
    double v = dot3(d, q) / det;
    if (v < 0.0 || u + v > 1.0) return 0;
    double tt = dot3(e2, q) / det;
    if (!(tt > 0.0)) return 0;
    *t = tt;
    double w = 1.0 - u - v;
    *bmin = fmin(u, fmin(v, w));
    return 1;
}

typedef struct {
    double t, t2, bmin;
    int64_t k;
    int64_t tests, nodes;
} orc_hit;

/* candidate triangle k of the FP64 ray (o, d) */
static void consider(const orc_mesh* m, int64_t k, const double* o, const double* d, orc_hit* h)
{
    double t, b;
    h->tests++;
    if (!tri_hit(m, k, o, d, &t, &b)) return;
    if (t < h->t || (t == h->t && k < h->k)) {
        if (h->k >= 0 && h->t < h->t2) h->t2 = h->t;
        h->t = t;
        h->k = k;
        h->bmin = b;
    } else if (t < h->t2) {
        h->t2 = t;
    }
}

static int slab(const orc_node* nd, const double* o, const double* d, double tmax, double* tenter)
{
    double t0 = 0.0, t1 = tmax;
    for (int c = 0; c < 3; ++c) {
        if (d[c] == 0.0) {
            if (o[c] < nd->lo[c] || o[c] > nd->hi[c]) return 0;
            continue;
        }
        double a = (nd->lo[c] - o[c]) / d[c], b = (nd->hi[c] - o[c]) / d[c];
        if (a > b) { double x = a; a = b; b = x; }
        if (a > t0) t0 = a;
        if (b < t1) t1 = b;
        if (t0 > t1) return 0;
    }
    *tenter = t0;
    return 1;
}

/* closest hit of the ray (o, d) skipping triangle `skip`; use_bvh = 0 brute
 * force, 1 median BVH. t2 is the runner-up candidate's t (INFINITY if none). */
static void closest(const orc_mesh* m, int use_bvh, const double* o, const double* d, int64_t skip, orc_hit* h)
{
    h->t = INFINITY;
    h->t2 = INFINITY;
    h->bmin = 0.0;
    h->k = -1;
    h->tests = h->nodes = 0;
    if (!use_bvh || !m->nodes) {
        for (int64_t k = 0; k < m->nt; ++k)
            if (k != skip) consider(m, k, o, d, h);
        return;
    }
    int64_t stack[256];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const orc_node* nd = &m->nodes[stack[--sp]];
        double te;
        h->nodes++;
        /* keep boxes up to 1e-5 beyond the best hit so the runner-up within 1e-6 is seen */
        double lim = isinf(h->t) ? INFINITY : h->t * (1.0 + 1e-5) + 1e-300;
        if (!slab(nd, o, d, lim, &te)) continue;
        if (nd->count > 0) {
            for (int64_t i = nd->first; i < nd->first + nd->count; ++i) {
                int64_t k = m->order[i];
                if (k != skip) consider(m, k, o, d, h);
            }
            continue;
        }
        /* near child first: push the far one first */
        const orc_node *L = &m->nodes[nd->left], *R = &m->nodes[nd->right];
        double tl = INFINITY, tr = INFINITY;
        int hl = slab(L, o, d, lim, &tl), hr = slab(R, o, d, lim, &tr);
        if (sp + 2 > 256) return; /* cannot happen for median trees below 2^128 leaves */
        if (hl && hr) {
            if (tl <= tr) { stack[sp++] = nd->right; stack[sp++] = nd->left; }
            else { stack[sp++] = nd->left; stack[sp++] = nd->right; }
        } else if (hl) {
            stack[sp++] = nd->left;
        } else if (hr) {
            stack[sp++] = nd->right;
        }
    }
}

int orc_closest_hit(const orc_mesh* m, int use_bvh, const double* o, const double* d, int64_t skip,
                    double* t, int64_t* tri, double* bmin, double* t2)
{
    orc_hit h;
    closest(m, use_bvh, o, d, skip, &h);
    *t = h.t;
    *tri = h.k;
    *bmin = h.bmin;
    *t2 = h.t2;
    return h.k >= 0;
}

/* ------------------------------------------------------------------ transport (Algorithm 2) */
/* Specular reflection d' = d - 2 (d.n) n and PEC field update E' = 2 (n.E) n - E
 * (tangential E reversed, normal E kept), for a unit normal n. */
static void reflect(const double* n, double* d, double* E1, double* E2)
{
    double dn = dot3(d, n), a = dot3(n, E1), b = dot3(n, E2);
    for (int c = 0; c < 3; ++c) {
        d[c] = d[c] - 2.0 * dn * n[c];
        E1[c] = 2.0 * a * n[c] - E1[c];
        E2[c] = 2.0 * b * n[c] - E2[c];
    }
}

void orc_reflect(const double* n, double* d, double* E1, double* E2) { reflect(n, d, E1, E2); }

typedef struct {
    int max_bounces;
    int po_mode;        /* 0 vector, 1 paper scalar */
    int phase_literal;  /* scalar mode only: L = 2 (k.o0 + R) */
    int require_escape;
    int use_bvh;
    int n_threads;
} orc_trace_opts;

typedef struct {
    const orc_mesh* m;
    const orc_frame* f;
    const orc_trace_opts* opt;
    const int64_t* ids;
    int64_t n;
    int32_t* hit_tri;  /* [n][B] original triangle index or -1 */
    double* hit_t;     /* [n][B] */
    int32_t* nb;       /* [n] bounces N */
    uint8_t* valid;    /* [n] */
    uint8_t* band;     /* [n] bit0 barycentric band, bit1 runner-up band */
    double* coef;      /* [n][4] HH, VV, HV, VH */
    double* Lpath;     /* [n] */
    double* bmin;      /* [n] smallest barycentric of the hits along the path (1 if no hit) */
    int64_t* counters; /* [2] per call: triangle tests, node visits */
    int64_t t_begin, t_end;
    int64_t tests, nodes;
} trace_job;

static void trace_one(trace_job* J, int64_t r)
{
    const orc_frame* f = J->f;
    const orc_trace_opts* opt = J->opt;
    const orc_mesh* m = J->m;
    const int B = opt->max_bounces;
    int64_t rid = J->ids ? J->ids[r] : r;
    int64_t i = rid % f->nu, j = rid / f->nu;
    /* the ray state, stored in FP32 between bounces */
    float o32[3], d32[3];
    orc_ray(f, i, j, o32, d32);
    double o[3] = {o32[0], o32[1], o32[2]}, d[3] = {d32[0], d32[1], d32[2]};
    const float eps32 = (float)f->eps;
    double Ev[3], Eh[3];
    for (int c = 0; c < 3; ++c) { Ev[c] = f->vhat[c]; Eh[c] = f->hhat[c]; }
    double ref = dot3(f->khat, o); /* k.o0 */
    double R = 0.0, L = 0.0, cos0 = 0.0;
    double cv[4] = {0, 0, 0, 0};
    float nf_last[3] = {0, 0, 0};
    int N = 0;
    uint8_t band = 0;
    double bmin_path = 1.0;
    int64_t skip = -1;
    for (int b = 0; b < B; ++b) {
        if (J->hit_tri) J->hit_tri[r * B + b] = -1;
        if (J->hit_t) J->hit_t[r * B + b] = 0.0;
    }
    for (int b = 0; b < B; ++b) {
        orc_hit h;
        for (int c = 0; c < 3; ++c) { o[c] = o32[c]; d[c] = d32[c]; }
        closest(m, opt->use_bvh, o, d, skip, &h);
        J->tests += h.tests;
        J->nodes += h.nodes;
        if (h.k < 0) break;
        if (h.bmin < 1e-6) band |= 1;
        if (h.bmin < bmin_path) bmin_path = h.bmin;
        if (h.t2 - h.t <= 1e-6 * h.t) band |= 2;
        /* next FP32 state: distance to the plane of the FP32 unit normal through
         * v0, hit point, reflection about n32 and the offset origin */
        const float* n32 = m->n32 + 3 * h.k;
        const double* v0 = m->v0 + 3 * h.k;
        double nd[3] = {n32[0], n32[1], n32[2]}, dv[3];
        for (int c = 0; c < 3; ++c) dv[c] = v0[c] - o[c];
        const double num = dot3(dv, nd), den = dot3(d, nd);
        const float t32 = den != 0.0 ? (float)(num / den) : (float)h.t;
        const float c32 = (float)den;
        const int front = den < 0.0; /* n32 faces the incoming ray */
        float x32[3], nf32[3];
        for (int c = 0; c < 3; ++c) {
            x32[c] = fmaf(t32, d32[c], o32[c]);
            nf32[c] = front ? n32[c] : -n32[c];
        }
        double x[3], nf[3], din[3];
        for (int c = 0; c < 3; ++c) {
            x[c] = x32[c];
            nf[c] = nf32[c];
            din[c] = d[c];
            nf_last[c] = nf32[c];
        }
        R += (double)t32;
        N += 1;
        if (J->hit_tri) J->hit_tri[r * B + b] = (int32_t)h.k;
        if (J->hit_t) J->hit_t[r * B + b] = (double)t32;
        const double dn = dot3(din, nd);
        if (N == 1) cos0 = dot3(nf, f->rhat);
        /* candidate contribution if this hit is the last one; the far-field
         * phase reference is the origin, toward the receiver: L = k.o0 + R - r_rx.x */
        L = ref + R - dot3(f->rx_rhat, x);
        {
            double adn = fabs(dn);
            double dS = adn > 0.0 ? f->dA / adn : 0.0;
            const double* Eq[2] = {Eh, Ev}; /* transmit H, transmit V */
            double W[2][3];
            for (int q = 0; q < 2; ++q) {
                double Hf[3], Jc[3];
                cross3(din, Eq[q], Hf);
                cross3(nf, Hf, Jc);
                for (int c = 0; c < 3; ++c) Jc[c] *= 2.0;
                double jr = dot3(Jc, f->rx_rhat);
                for (int c = 0; c < 3; ++c) W[q][c] = dS * (Jc[c] - jr * f->rx_rhat[c]);
            }
            cv[0] = dot3(W[0], f->rx_hhat); /* HH: receive H, transmit H */
            cv[1] = dot3(W[1], f->rx_vhat); /* VV */
            cv[2] = dot3(W[1], f->rx_hhat); /* HV: receive H, transmit V */
            cv[3] = dot3(W[0], f->rx_vhat); /* VH: receive V, transmit H */
        }
        {
            double dd[3] = {din[0], din[1], din[2]};
            reflect(nd, dd, Ev, Eh); /* PEC field update in FP64 about the facet's normal */
        }
        for (int c = 0; c < 3; ++c) {
            d32[c] = fmaf(-2.0f * c32, n32[c], d32[c]);
            o32[c] = fmaf(eps32, nf32[c], x32[c]);
        }
        skip = h.k;
    }
    for (int c = 0; c < 3; ++c) { o[c] = o32[c]; d[c] = d32[c]; }
    int valid = N >= 1;
    if (valid && opt->require_escape && N == B) {
        orc_hit h;
        closest(m, opt->use_bvh, o, d, skip, &h);
        J->tests += h.tests;
        J->nodes += h.nodes;
        if (h.k >= 0) valid = 0;
    }
    if (valid && f->bistatic) {
        /* visibility of the last hit from the receiver: the receiver lies on the
         * side of the oriented normal (sign of the exact dot product of the FP32
         * vectors), and the ray from the offset origin toward it meets no
         * triangle (the one just hit is skipped) */
        double rxd[3] = {f->rx_r32[0], f->rx_r32[1], f->rx_r32[2]};
        double nfl[3] = {nf_last[0], nf_last[1], nf_last[2]};
        int sees = dot3(nfl, rxd) > 0.0;
        if (sees) {
            orc_hit h;
            closest(m, opt->use_bvh, o, rxd, skip, &h);
            J->tests += h.tests;
            J->nodes += h.nodes;
            sees = h.k < 0;
        }
        if (!sees) valid = 0;
    }
    if (opt->po_mode == 1) {
        double s = (N & 1) ? -1.0 : 1.0; /* Gamma^N, Gamma = -1 */
        double c = -(2.0 * f->dA * cos0 * s);
        cv[0] = c; cv[1] = c; cv[2] = 0.0; cv[3] = 0.0;
        if (opt->phase_literal) L = 2.0 * (ref + R);
    }
    if (J->nb) J->nb[r] = N;
    if (J->valid) J->valid[r] = (uint8_t)valid;
    if (J->band) J->band[r] = band;
    if (J->coef)
        for (int p = 0; p < 4; ++p) J->coef[4 * r + p] = valid ? cv[p] : 0.0;
    if (J->Lpath) J->Lpath[r] = valid ? L : 0.0;
    if (J->bmin) J->bmin[r] = bmin_path;
}

static void* trace_worker(void* arg)
{
    trace_job* J = (trace_job*)arg;
    for (int64_t r = J->t_begin; r < J->t_end; ++r) trace_one(J, r);
    return NULL;
}

/* Trace rays `ids` (NULL: every ray of the frame, n = nu*nv). Outputs may be NULL. */
int orc_trace(const orc_mesh* m, const orc_frame* f, const orc_trace_opts* opt, const int64_t* ids, int64_t n,
              int32_t* hit_tri, double* hit_t, int32_t* nb, uint8_t* valid, uint8_t* band, double* coef,
              double* Lpath, double* bmin, int64_t* counters)
{
    if (!m || !f || !opt || opt->max_bounces < 1 || n < 0) return -1;
    int T = opt->n_threads > 0 ? opt->n_threads : 1;
    if (T > 256) T = 256;
    if (n < T) T = n > 0 ? (int)n : 1;
    trace_job jobs[256];
    pthread_t th[256];
    for (int t = 0; t < T; ++t) {
        trace_job* J = &jobs[t];
        memset(J, 0, sizeof(*J));
        J->m = m; J->f = f; J->opt = opt; J->ids = ids; J->n = n;
        J->hit_tri = hit_tri; J->hit_t = hit_t; J->nb = nb; J->valid = valid; J->band = band;
        J->coef = coef; J->Lpath = Lpath; J->bmin = bmin;
        J->t_begin = n * t / T;
        J->t_end = n * (t + 1) / T;
    }
    for (int t = 1; t < T; ++t) pthread_create(&th[t], NULL, trace_worker, &jobs[t]);
    trace_worker(&jobs[0]);
    for (int t = 1; t < T; ++t) pthread_join(th[t], NULL);
    if (counters) {
        counters[0] = counters[1] = 0;
        for (int t = 0; t < T; ++t) { counters[0] += jobs[t].tests; counters[1] += jobs[t].nodes; }
    }
    return 0;
}

/* ------------------------------------------------------------------ PO sum (Eq. po_sum / em6) */
/* E[f][p] = (-j k / 4 pi) sum_r coef[r][p] exp(-j k L_r), summed in ray order in FP64.
 * E is written as [n_freq][4][2] (re, im); rcs_dbsm as [n_freq][4] (10 log10 4 pi |E|^2). */
int orc_po(const double* coef, const double* Lpath, const uint8_t* valid, int64_t n, const double* freq,
           int64_t n_freq, double* E, double* rcs_dbsm)
{
    if (!coef || !Lpath || !freq || !E || n < 0) return -1;
    for (int64_t fi = 0; fi < n_freq; ++fi) {
        double k = 2.0 * ORC_PI * freq[fi] / ORC_C0;
        double sr[4] = {0, 0, 0, 0}, si[4] = {0, 0, 0, 0};
        for (int64_t r = 0; r < n; ++r) {
            if (valid && !valid[r]) continue;
            double ph = k * Lpath[r];
            double c = cos(ph), s = -sin(ph);
            for (int p = 0; p < 4; ++p) {
                sr[p] += coef[4 * r + p] * c;
                si[p] += coef[4 * r + p] * s;
            }
        }
        double pre = k / (4.0 * ORC_PI); /* -j pre (sr + j si) = pre (si - j sr) */
        for (int p = 0; p < 4; ++p) {
            double er = pre * si[p], ei = -pre * sr[p];
            E[(fi * 4 + p) * 2 + 0] = er;
            E[(fi * 4 + p) * 2 + 1] = ei;
            if (rcs_dbsm) rcs_dbsm[fi * 4 + p] = 10.0 * log10(4.0 * ORC_PI * (er * er + ei * ei));
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ Mie series, PEC sphere */
/* Monostatic backscatter efficiency sigma / (pi a^2) of a perfectly conducting
 * sphere of size parameter x = k a, from the Riccati-Bessel series
 *   Q_b = x^-2 | sum_n (2n+1) (-1)^n (a_n - b_n) |^2,
 *   a_n = psi_n'(x) / xi_n'(x),  b_n = psi_n(x) / xi_n(x),  xi_n = psi_n - i chi_n,
 * psi_n from the downward-recurred logarithmic derivative, chi_n by upward
 * recurrence, terms to n = x + 4 x^(1/3) + 10. */
double orc_mie_pec_backscatter(double x)
{
    if (!(x > 0.0)) return 0.0;
    int nmax = (int)(x + 4.0 * cbrt(x) + 10.0);
    int nstart = (int)fmax((double)nmax, x) + 16;
    double* Dn = (double*)malloc(sizeof(double) * (size_t)(nstart + 1));
    Dn[nstart] = 0.0;
    for (int n = nstart; n >= 1; --n) Dn[n - 1] = (double)n / x - 1.0 / (Dn[n] + (double)n / x);
    double psi_m1 = sin(x);  /* psi_0 */
    double chi_m1 = cos(x);  /* chi_0 */
    double chi_m2 = -sin(x); /* chi_{-1} */
    double Sr = 0.0, Si = 0.0;
    for (int n = 1; n <= nmax; ++n) {
        double psi = psi_m1 / (Dn[n] + (double)n / x);
        double chi = (2.0 * n - 1.0) / x * chi_m1 - chi_m2;
        double dpsi = psi_m1 - (double)n / x * psi;
        double dchi = chi_m1 - (double)n / x * chi;
        /* a_n = dpsi / (dpsi - i dchi), b_n = psi / (psi - i chi) */
        double den_a = dpsi * dpsi + dchi * dchi, den_b = psi * psi + chi * chi;
        double ar = dpsi * dpsi / den_a, ai = dpsi * dchi / den_a;
        double br = psi * psi / den_b, bi = psi * chi / den_b;
        double w = (2.0 * n + 1.0) * ((n & 1) ? -1.0 : 1.0);
        Sr += w * (ar - br);
        Si += w * (ai - bi);
        psi_m1 = psi;
        chi_m2 = chi_m1;
        chi_m1 = chi;
    }
    free(Dn);
    return (Sr * Sr + Si * Si) / (x * x);
}
