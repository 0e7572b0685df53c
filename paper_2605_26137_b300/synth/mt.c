/*
 * Marching tetrahedra over a sampled signed distance field: the test-fixture
 * mesher for the seeded synthetic assets (dense "high-poly" and coarse
 * "low-poly" surfaces extracted from one SDF, as the geometry stage of the
 * paper does with marching cubes in its post-processing section).
 *
 * This is input generation only; it holds none of the baking arithmetic and
 * is shared by the CUDA path's tests and by the oracle's tests.
 *
 * Each grid cube is split into six tetrahedra along its main diagonal (the
 * Kuhn / Freudenthal split), which tiles space consistently, so the extracted
 * surface is watertight.  Every tetrahedron edge joins two cube corners whose
 * offset bit-sets are nested, so an edge is named by its lower grid node and a
 * direction mask in 1..7; vertices are welded on that key, plane by plane.
 * The triangle case table is derived at start-up from the geometry of the
 * canonical cube (no stored table).
 *
 * Sign convention: a node is inside when f < 0.  Triangles are wound so their
 * normal points from inside to outside.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* tetrahedron t: corners (as xyz offset bit-sets) {0, 1<<a0, (1<<a0)|(1<<a1), 7} */
static int g_tet[6][4];
/* case table: for tet t and inside-mask c, up to 2 triangles of 3 edges, each
 * edge a pair of tet-local vertex slots */
static int g_ntri[6][16];
static int g_tri[6][16][2][3][2];
static int g_ready = 0;

static void corner_pos(int m, double p[3]) {
    p[0] = (double)(m & 1);
    p[1] = (double)((m >> 1) & 1);
    p[2] = (double)((m >> 2) & 1);
}

static void emit_oriented(int t, int c, int k, int ea[3][2], const double in_c[3], const double out_c[3]) {
    double q[3][3];
    for (int i = 0; i < 3; ++i) {
        double a[3], b[3];
        corner_pos(g_tet[t][ea[i][0]], a);
        corner_pos(g_tet[t][ea[i][1]], b);
        for (int j = 0; j < 3; ++j) q[i][j] = 0.5 * (a[j] + b[j]);
    }
    double u[3], v[3], n[3];
    for (int j = 0; j < 3; ++j) { u[j] = q[1][j] - q[0][j]; v[j] = q[2][j] - q[0][j]; }
    n[0] = u[1] * v[2] - u[2] * v[1];
    n[1] = u[2] * v[0] - u[0] * v[2];
    n[2] = u[0] * v[1] - u[1] * v[0];
    double dir = 0.0;
    for (int j = 0; j < 3; ++j) dir += n[j] * (out_c[j] - in_c[j]);
    int order[3] = {0, 1, 2};
    if (dir < 0.0) { order[1] = 2; order[2] = 1; }
    for (int i = 0; i < 3; ++i) {
        g_tri[t][c][k][i][0] = ea[order[i]][0];
        g_tri[t][c][k][i][1] = ea[order[i]][1];
    }
}

static void build_tables(void) {
    if (g_ready) return;
    int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int t = 0; t < 6; ++t) {
        g_tet[t][0] = 0;
        g_tet[t][1] = 1 << perms[t][0];
        g_tet[t][2] = (1 << perms[t][0]) | (1 << perms[t][1]);
        g_tet[t][3] = 7;
    }
    for (int t = 0; t < 6; ++t) {
        for (int c = 0; c < 16; ++c) {
            int ins[4], outs[4], ni = 0, no = 0;
            for (int s = 0; s < 4; ++s) {
                if (c & (1 << s)) ins[ni++] = s; else outs[no++] = s;
            }
            double in_c[3] = {0, 0, 0}, out_c[3] = {0, 0, 0};
            for (int s = 0; s < ni; ++s) { double p[3]; corner_pos(g_tet[t][ins[s]], p); for (int j = 0; j < 3; ++j) in_c[j] += p[j] / ni; }
            for (int s = 0; s < no; ++s) { double p[3]; corner_pos(g_tet[t][outs[s]], p); for (int j = 0; j < 3; ++j) out_c[j] += p[j] / no; }
            g_ntri[t][c] = 0;
            if (ni == 0 || ni == 4) continue;
            if (ni == 1 || ni == 3) {
                int apex = (ni == 1) ? ins[0] : outs[0];
                int *others = (ni == 1) ? outs : ins;
                int ea[3][2];
                for (int i = 0; i < 3; ++i) { ea[i][0] = apex; ea[i][1] = others[i]; }
                emit_oriented(t, c, 0, ea, in_c, out_c);
                g_ntri[t][c] = 1;
            } else {
                /* quad on edges (a,c) (a,d) (b,d) (b,c), a,b inside, c,d outside */
                int a = ins[0], b = ins[1], cc = outs[0], d = outs[1];
                int e0[3][2] = {{a, cc}, {a, d}, {b, d}};
                int e1[3][2] = {{a, cc}, {b, d}, {b, cc}};
                emit_oriented(t, c, 0, e0, in_c, out_c);
                emit_oriented(t, c, 1, e1, in_c, out_c);
                g_ntri[t][c] = 2;
            }
        }
    }
    g_ready = 1;
}

typedef struct {
    float *v; int64_t nv, cap_v;
    int32_t *f; int64_t nf, cap_f;
} mesh_buf;

static int push_vertex(mesh_buf *m, float x, float y, float z) {
    if (m->nv == m->cap_v) {
        int64_t nc = m->cap_v ? m->cap_v * 2 : 1 << 16;
        float *nv = (float *)realloc(m->v, (size_t)nc * 3 * sizeof(float));
        if (!nv) return -1;
        m->v = nv; m->cap_v = nc;
    }
    m->v[m->nv * 3 + 0] = x; m->v[m->nv * 3 + 1] = y; m->v[m->nv * 3 + 2] = z;
    m->nv++;
    return 0;
}

static int push_face(mesh_buf *m, int32_t a, int32_t b, int32_t c) {
    if (m->nf == m->cap_f) {
        int64_t nc = m->cap_f ? m->cap_f * 2 : 1 << 16;
        int32_t *nf = (int32_t *)realloc(m->f, (size_t)nc * 3 * sizeof(int32_t));
        if (!nf) return -1;
        m->f = nf; m->cap_f = nc;
    }
    m->f[m->nf * 3 + 0] = a; m->f[m->nf * 3 + 1] = b; m->f[m->nf * 3 + 2] = c;
    m->nf++;
    return 0;
}

/*
 * f: node values, layout f[(k*ny + j)*nx + i]; node (i,j,k) sits at
 * (x0 + i*h, y0 + j*h, z0 + k*h).  On success returns 0 and hands out malloc'd
 * arrays (release with mt_free).  Returns -1 on allocation failure.
 */
int mt_extract(const float *f, int nx, int ny, int nz, double x0, double y0, double z0, double h,
               float **out_v, int64_t *out_nv, int32_t **out_f, int64_t *out_nf) {
    build_tables();
    mesh_buf m = {0};
    size_t plane = (size_t)nx * (size_t)ny * 7;
    int32_t *cur = (int32_t *)malloc(plane * sizeof(int32_t));
    int32_t *nxt = (int32_t *)malloc(plane * sizeof(int32_t));
    if (!cur || !nxt) { free(cur); free(nxt); return -1; }
    memset(cur, 0xff, plane * sizeof(int32_t));
    memset(nxt, 0xff, plane * sizeof(int32_t));
    int err = 0;
    for (int k = 0; k + 1 < nz && !err; ++k) {
        for (int j = 0; j + 1 < ny && !err; ++j) {
            for (int i = 0; i + 1 < nx && !err; ++i) {
                float cv[8];
                int nin = 0;
                for (int m8 = 0; m8 < 8; ++m8) {
                    int ii = i + (m8 & 1), jj = j + ((m8 >> 1) & 1), kk = k + ((m8 >> 2) & 1);
                    cv[m8] = f[((size_t)kk * ny + jj) * nx + ii];
                    nin += cv[m8] < 0.0f;
                }
                if (nin == 0 || nin == 8) continue;
                for (int t = 0; t < 6 && !err; ++t) {
                    int c = 0;
                    for (int s = 0; s < 4; ++s) c |= (cv[g_tet[t][s]] < 0.0f) << s;
                    for (int tr = 0; tr < g_ntri[t][c]; ++tr) {
                        int32_t vid[3];
                        for (int e = 0; e < 3; ++e) {
                            int ma = g_tet[t][g_tri[t][c][tr][e][0]];
                            int mb = g_tet[t][g_tri[t][c][tr][e][1]];
                            int lo = (ma & mb) == ma ? ma : mb; /* nested corner sets */
                            int hi = lo == ma ? mb : ma;
                            int dir = hi & ~lo;
                            int li = i + (lo & 1), lj = j + ((lo >> 1) & 1), lz = (lo >> 2) & 1;
                            int32_t *map = lz ? nxt : cur;
                            size_t key = ((size_t)lj * nx + li) * 7 + (size_t)(dir - 1);
                            if (map[key] < 0) {
                                double fa = cv[lo], fb = cv[hi];
                                double s = fa / (fa - fb);
                                double pa[3] = {x0 + (i + (lo & 1)) * h, y0 + (j + ((lo >> 1) & 1)) * h, z0 + (k + ((lo >> 2) & 1)) * h};
                                double pb[3] = {x0 + (i + (hi & 1)) * h, y0 + (j + ((hi >> 1) & 1)) * h, z0 + (k + ((hi >> 2) & 1)) * h};
                                if (push_vertex(&m, (float)(pa[0] + s * (pb[0] - pa[0])),
                                                (float)(pa[1] + s * (pb[1] - pa[1])),
                                                (float)(pa[2] + s * (pb[2] - pa[2])))) { err = 1; break; }
                                map[key] = (int32_t)(m.nv - 1);
                            }
                            vid[e] = map[key];
                        }
                        if (err) break;
                        if (push_face(&m, vid[0], vid[1], vid[2])) { err = 1; break; }
                    }
                }
            }
        }
        int32_t *tmp = cur; cur = nxt; nxt = tmp;
        memset(nxt, 0xff, plane * sizeof(int32_t));
    }
    free(cur); free(nxt);
    if (err) { free(m.v); free(m.f); return -1; }
    *out_v = m.v; *out_nv = m.nv; *out_f = m.f; *out_nf = m.nf;
    return 0;
}

void mt_free(void *p) { free(p); }
