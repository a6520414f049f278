/* Plain C user of the boundary: include/sbr.h and libsbr.so only.
 * Builds a square PEC plate (side 1 m, 2 x m x m triangles) in the z = 0 plane,
 * traces it at the aspects given on the command line (az el pairs, degrees),
 * integrates HH and VV at 10 GHz and prints one line per aspect:
 *   az el rcs_hh_dbsm rcs_vv_dbsm valid_rays
 * Exit status: 0 on success, 1 on any library error (message on stderr). */
#include <stdio.h>
#include <stdlib.h>

#include "sbr.h"

static int check(sbr_ctx* c, int rc, const char* what)
{
    if (rc != SBR_OK) fprintf(stderr, "%s failed (%d): %s\n", what, rc, sbr_last_error(c));
    return rc != SBR_OK;
}

int main(int argc, char** argv)
{
    const int m = 8;
    const int nv = (m + 1) * (m + 1), nt = 2 * m * m;
    float* xyz = (float*)malloc(sizeof(float) * 3 * nv);
    int32_t* tri = (int32_t*)malloc(sizeof(int32_t) * 3 * nt);
    /* vertex i (m + 1) + j at (x_i, y_j), x_i = y_i = -1/2 + i / m; triangles (p, q, p + 1), (q, q + 1, p + 1) */
    for (int i = 0; i <= m; ++i)
        for (int j = 0; j <= m; ++j) {
            float* p = xyz + 3 * (i * (m + 1) + j);
            p[0] = (float)(-0.5 + (double)i / m);
            p[1] = (float)(-0.5 + (double)j / m);
            p[2] = 0.f;
        }
    int t = 0;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            const int p = i * (m + 1) + j, q = (i + 1) * (m + 1) + j;
            tri[3 * t] = p; tri[3 * t + 1] = q; tri[3 * t + 2] = p + 1; ++t;
            tri[3 * t] = q; tri[3 * t + 1] = q + 1; tri[3 * t + 2] = p + 1; ++t;
        }
    const int n_ang = (argc - 1) / 2;
    if (n_ang < 1) {
        fprintf(stderr, "usage: %s az el [az el ...]\n", argv[0]);
        return 1;
    }
    double* ang = (double*)malloc(sizeof(double) * 2 * n_ang);
    for (int a = 0; a < 2 * n_ang; ++a) ang[a] = atof(argv[1 + a]);

    sbr_ctx* ctx = NULL;
    if (sbr_create(&ctx, 0, NULL) != SBR_OK) {
        fprintf(stderr, "sbr_create failed: %s\n", sbr_last_error(NULL));
        return 1;
    }
    int bad = check(ctx, sbr_load_mesh(ctx, xyz, nv, tri, nt, 0), "sbr_load_mesh");
    sbr_trace_opts opt = {0};
    opt.window_m = 1.3;
    sbr_trace_stats st;
    const double freq = 10e9;
    if (!bad)
        bad = check(ctx, sbr_trace(ctx, ang, n_ang, sbr_spacing_for(freq, 10.0), 0.05, 1, &opt, &st), "sbr_trace");
    double* E = (double*)malloc(sizeof(double) * 2 * 2 * n_ang);
    double* rcs = (double*)malloc(sizeof(double) * 2 * n_ang);
    if (!bad)
        bad = check(ctx, sbr_po_integrate(ctx, &freq, 1, SBR_POL_HH | SBR_POL_VV, SBR_PO_VECTOR, E, rcs, 0),
                    "sbr_po_integrate");
    for (int a = 0; a < n_ang && !bad; ++a)
        printf("%.17g %.17g %.17g %.17g %lld\n", ang[2 * a], ang[2 * a + 1], rcs[2 * a], rcs[2 * a + 1],
               (long long)st.valid_rays);
    sbr_destroy(ctx);
    free(xyz);
    free(tri);
    free(ang);
    free(E);
    free(rcs);
    return bad;
}
