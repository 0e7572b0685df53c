/*
 * FP64 CPU oracle for tangent-space normal baking (Sec. 6.4, "Normal Map
 * Baking").  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * CPU-baseline leg of the benchmark call it; the product path never does.
 * It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes, step by step, in the order Sec. 6.4 lists them:
 *   1. area-weighted smooth vertex normals of both meshes;
 *   2. the low-poly mesh rasterised into its own UV space: per texel the
 *      owning low face and barycentrics (exact fixed-point predicates);
 *   3. per-face tangent frames from the UV gradients, and the
 *      "degenerate UV" reliability flag;
 *   4. per ray texel: origin p = sum b_i v_i, direction d = normalize(sum b_i n_i),
 *      the closest hit (minimum |t|, |t| <= max_dist) of the line p + t d
 *      against every high-poly triangle (brute force, or a median-split BVH
 *      that is pinned bit-for-bit to brute force); or, as Sec. 6.4 words it,
 *      the closest point of the high surface to p (same two searches);
 *   5. the hit's barycentric smooth normal projected into the texel frame;
 *   6. RGB8 encoding and gutter dilation;
 *   7. the baking loss mean(t^2) + lambda*mean(1 - n_hit . d) over hit texels
 *      and its analytic gradient with respect to the low-poly positions;
 *   8. hidden-face removal (Sec. 6.2): per-face visibility from orthographic
 *      views around the mesh, then the normal-gated exterior flood fill.
 *
 * Readings of points the paper leaves open are stated where they are used.
 * Everything is double precision except the UV snapping, which is exact
 * integer arithmetic by definition (texel coordinates * 256, rounded half
 * away from zero).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ vectors */
typedef struct { double x, y, z; } d3;
static d3 mk(double x, double y, double z) { d3 r = {x, y, z}; return r; }
static d3 add(d3 a, d3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static d3 sub(d3 a, d3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static d3 scl(d3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static d3 cross(d3 a, d3 b) { return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static double norm(d3 a) { return sqrt(dot(a, a)); }
static d3 normalize(d3 a) { double n = norm(a); return n > 0 ? scl(a, 1.0 / n) : a; }
static d3 ldf(const float *p, int64_t i) { return mk(p[3 * i], p[3 * i + 1], p[3 * i + 2]); }
static d3 ldd(const double *p, int64_t i) { return mk(p[3 * i], p[3 * i + 1], p[3 * i + 2]); }
static void std3(double *p, int64_t i, d3 v) { p[3 * i] = v.x; p[3 * i + 1] = v.y; p[3 * i + 2] = v.z; }
static double comp(d3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

/* ------------------------------------------------- 1. vertex normals (Sec. 6.4)
 * "smooth normal": n_i = normalize(sum over faces f containing i of
 * (v1 - v0) x (v2 - v0)); the unnormalised cross product weights each face
 * by its area (reading). */
void or_vertex_normals(const float *V, int64_t nv, const int32_t *F, int64_t nf, double *N) {
    memset(N, 0, sizeof(double) * 3 * (size_t)nv);
    for (int64_t f = 0; f < nf; ++f) {
        int32_t a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
        d3 va = ldf(V, a), vb = ldf(V, b), vc = ldf(V, c);
        d3 n = cross(sub(vb, va), sub(vc, va));
        for (int k = 0; k < 3; ++k) {
            int32_t i = F[3 * f + k];
            std3(N, i, add(ldd(N, i), n));
        }
    }
    for (int64_t i = 0; i < nv; ++i) std3(N, i, normalize(ldd(N, i)));
}

/* ------------------------------------------------- 2. UV-space raster (Sec. 6.4)
 * Reading of the rasterisation of the low-poly mesh in its own UV layout:
 *  - texel (x, y) has centre (x + 1/2, y + 1/2) in texel units, x = u*W,
 *    y = v*H (v not flipped);
 *  - UVs are snapped to 1/256 texel: X = round_half_away(u * W * 256);
 *  - owner: the lowest-id face whose closed triangle contains the centre;
 *  - otherwise (conservative coverage) among faces whose triangle overlaps the
 *    texel square with positive area, the one nearest the centre, with squared
 *    distances compared at a resolution of 2^-16 (1/256 texel)^2 units
 *    (floor), ties to the lowest id; barycentrics are those of the closest
 *    point of that triangle;
 *  - zero-area faces own nothing; faces with |UV area| < 1e-4 texel^2
 *    (|2*area| <= 13 in snapped units) are flagged "degenerate UV".
 */
int64_t or_snap(float u, int W) {
    double x = (double)u * (double)W * 256.0; /* exact: 24-bit mantissa x <= 22-bit integer */
    return x >= 0 ? (int64_t)floor(x + 0.5) : -(int64_t)floor(-x + 0.5);
}

typedef struct { int64_t X[3], Y[3], a2; } uvtri;

static void load_uvtri(const float *uv, int64_t f, int W, int H, uvtri *t) {
    for (int k = 0; k < 3; ++k) {
        t->X[k] = or_snap(uv[6 * f + 2 * k], W);
        t->Y[k] = or_snap(uv[6 * f + 2 * k + 1], H);
    }
    t->a2 = (t->X[1] - t->X[0]) * (t->Y[2] - t->Y[0]) - (t->Y[1] - t->Y[0]) * (t->X[2] - t->X[0]);
}

static int64_t orient2(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy) {
    return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
}

/* e[i] = twice the signed area opposite vertex i; inside closed triangle iff
 * all e[i] have the sign of a2 or are zero */
static int uv_inside(const uvtri *t, int64_t cx, int64_t cy, int64_t e[3]) {
    if (t->a2 == 0) return 0;
    e[0] = orient2(t->X[1], t->Y[1], t->X[2], t->Y[2], cx, cy);
    e[1] = orient2(t->X[2], t->Y[2], t->X[0], t->Y[0], cx, cy);
    e[2] = orient2(t->X[0], t->Y[0], t->X[1], t->Y[1], cx, cy);
    if (t->a2 > 0) return e[0] >= 0 && e[1] >= 0 && e[2] >= 0;
    return e[0] <= 0 && e[1] <= 0 && e[2] <= 0;
}

/* interiors of the triangle and of the square [sx, sx+256] x [sy, sy+256]
 * intersect iff no axis from either polygon's edge normals separates them */
static int uv_overlap(const uvtri *t, int64_t sx, int64_t sy) {
    if (t->a2 == 0) return 0;
    int64_t mnx = t->X[0], mxx = t->X[0], mny = t->Y[0], mxy = t->Y[0];
    for (int k = 1; k < 3; ++k) {
        if (t->X[k] < mnx) mnx = t->X[k];
        if (t->X[k] > mxx) mxx = t->X[k];
        if (t->Y[k] < mny) mny = t->Y[k];
        if (t->Y[k] > mxy) mxy = t->Y[k];
    }
    if (mxx <= sx || mnx >= sx + 256 || mxy <= sy || mny >= sy + 256) return 0;
    int64_t cxs[4] = {sx, sx + 256, sx, sx + 256}, cys[4] = {sy, sy, sy + 256, sy + 256};
    for (int k = 0; k < 3; ++k) {
        int a = k, b = (k + 1) % 3, c = (k + 2) % 3;
        int64_t nx = -(t->Y[b] - t->Y[a]), ny = t->X[b] - t->X[a];
        int64_t pe = nx * t->X[a] + ny * t->Y[a];
        int64_t po = nx * t->X[c] + ny * t->Y[c];
        int64_t tmn = pe < po ? pe : po, tmx = pe < po ? po : pe;
        int64_t smn = 0, smx = 0;
        for (int q = 0; q < 4; ++q) {
            int64_t p = nx * cxs[q] + ny * cys[q];
            if (q == 0 || p < smn) smn = p;
            if (q == 0 || p > smx) smx = p;
        }
        if (smx <= tmn || smn >= tmx) return 0;
    }
    return 1;
}

/* squared distance from (cx,cy) to edge k of t, quantised: floor(d^2 * 65536)
 * in snapped units; UINT64_MAX when d > 256 units (one texel).  Also returns
 * the closest point's parameter along the edge. */
static uint64_t edge_qdist(const uvtri *t, int k, int64_t cx, int64_t cy, double *param) {
    int a = k, b = (k + 1) % 3;
    int64_t wx = cx - t->X[a], wy = cy - t->Y[a];
    int64_t dx = t->X[b] - t->X[a], dy = t->Y[b] - t->Y[a];
    int64_t wd = wx * dx + wy * dy, dd = dx * dx + dy * dy;
    unsigned __int128 num, den;
    if (dd == 0 || wd <= 0) {
        num = (unsigned __int128)(wx * wx + wy * wy); den = 1; *param = 0.0;
    } else if (wd >= dd) {
        int64_t ux = cx - t->X[b], uy = cy - t->Y[b];
        num = (unsigned __int128)(ux * ux + uy * uy); den = 1; *param = 1.0;
    } else {
        int64_t cr = wx * dy - wy * dx;
        unsigned __int128 c2 = (unsigned __int128)(cr < 0 ? -cr : cr);
        num = c2 * c2; den = (unsigned __int128)dd; *param = (double)wd / (double)dd;
    }
    if (num > den * 65536u) return UINT64_MAX;
    return (uint64_t)((num * 65536u) / den);
}

static uint64_t tri_qdist(const uvtri *t, int64_t cx, int64_t cy, int *best_edge, double *best_param) {
    uint64_t best = UINT64_MAX;
    *best_edge = -1;
    for (int k = 0; k < 3; ++k) {
        double p;
        uint64_t q = edge_qdist(t, k, cx, cy, &p);
        if (q < best) { best = q; *best_edge = k; *best_param = p; }
    }
    return best;
}

#define KEY_NONE UINT64_MAX
#define KEY_CONSERVATIVE (1ull << 63)

static uint64_t texel_key(const uvtri *t, int64_t f, int x, int y) {
    int64_t cx = 256 * (int64_t)x + 128, cy = 256 * (int64_t)y + 128, e[3];
    if (uv_inside(t, cx, cy, e)) return (uint64_t)f;
    if (uv_overlap(t, 256 * (int64_t)x, 256 * (int64_t)y)) {
        int be; double bp;
        uint64_t q = tri_qdist(t, cx, cy, &be, &bp);
        if (q == UINT64_MAX) return KEY_NONE; /* cannot happen for an overlapping square */
        return KEY_CONSERVATIVE | (q << 31) | (uint64_t)f;
    }
    return KEY_NONE;
}

static int64_t fdiv(int64_t a, int64_t b) { int64_t q = a / b; if ((a % b != 0) && ((a < 0) != (b < 0))) --q; return q; }

/* face[H*W] (-1 empty), bary[H*W*3], a2[nf]; brute != 0 evaluates every
 * (texel, face) pair, otherwise only texels within one texel of each face's
 * bounding box (the predicates are identical). */
int or_raster(const float *uv, int64_t nf, int W, int H, int brute, int32_t *face, double *bary, int64_t *a2_out) {
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W * H);
    if (!key) return -1;
    for (int64_t i = 0; i < (int64_t)W * H; ++i) key[i] = KEY_NONE;
    for (int64_t f = 0; f < nf; ++f) {
        uvtri t;
        load_uvtri(uv, f, W, H, &t);
        if (a2_out) a2_out[f] = t.a2;
        int x0 = 0, x1 = W - 1, y0 = 0, y1 = H - 1;
        if (!brute) {
            int64_t mnx = t.X[0], mxx = t.X[0], mny = t.Y[0], mxy = t.Y[0];
            for (int k = 1; k < 3; ++k) {
                if (t.X[k] < mnx) mnx = t.X[k];
                if (t.X[k] > mxx) mxx = t.X[k];
                if (t.Y[k] < mny) mny = t.Y[k];
                if (t.Y[k] > mxy) mxy = t.Y[k];
            }
            int64_t a = fdiv(mnx, 256) - 1, b = fdiv(mxx, 256) + 1, c = fdiv(mny, 256) - 1, d = fdiv(mxy, 256) + 1;
            x0 = a < 0 ? 0 : (int)(a > W - 1 ? W : a);
            x1 = b > W - 1 ? W - 1 : (int)b;
            y0 = c < 0 ? 0 : (int)(c > H - 1 ? H : c);
            y1 = d > H - 1 ? H - 1 : (int)d;
        }
        for (int y = y0; y <= y1; ++y)
            for (int x = x0; x <= x1; ++x) {
                uint64_t k = texel_key(&t, f, x, y);
                if (k < key[(int64_t)y * W + x]) key[(int64_t)y * W + x] = k;
            }
    }
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t i = (int64_t)y * W + x;
            uint64_t k = key[i];
            if (k == KEY_NONE) { face[i] = -1; bary[3 * i] = bary[3 * i + 1] = bary[3 * i + 2] = 0.0; continue; }
            int64_t f = (int64_t)(k & 0x7fffffffull);
            face[i] = (int32_t)f;
            uvtri t;
            load_uvtri(uv, f, W, H, &t);
            int64_t cx = 256 * (int64_t)x + 128, cy = 256 * (int64_t)y + 128, e[3];
            if (!(k & KEY_CONSERVATIVE)) {
                uv_inside(&t, cx, cy, e);
                for (int q = 0; q < 3; ++q) bary[3 * i + q] = (double)e[q] / (double)t.a2;
            } else {
                int be; double bp = 0.0;
                tri_qdist(&t, cx, cy, &be, &bp);
                double b3[3] = {0, 0, 0};
                b3[be] = 1.0 - bp;
                b3[(be + 1) % 3] = bp;
                for (int q = 0; q < 3; ++q) bary[3 * i + q] = b3[q];
            }
        }
    free(key);
    return 0;
}

/* ------------------------------------------------- 3. tangent frames (Sec. 6.4)
 * The paper gives no tangent rule (reading): per face the UV-gradient
 * tangent T_f = dp/du and bitangent B_f = dp/dv of the affine map from snapped
 * UVs to positions; per corner T_f is Gram-Schmidt orthonormalised against
 * the corner's vertex normal; the handedness w = sign((n_0 x T_f) . B_f) is
 * taken from corner 0.  Faces with |UV area| < 1e-4 texel^2 are unreliable
 * ("degenerate UV" filter): their output normal is (0,0,1) and their corner
 * tangents come from the Duff et al. 2017 orthonormal basis of the normal. */
static d3 onb_tangent(d3 n) {
    double s = n.z >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (s + n.z);
    double b = n.x * n.y * a;
    return mk(1.0 + s * n.x * n.x * a, s * b, -s * n.x);
}

void or_face_frames(const float *V, const int32_t *F, int64_t nf, const float *uv, int W, int H,
                    const double *N, double *T /*[nf*3*3]*/, double *wsign /*[nf]*/, uint8_t *degen /*[nf]*/) {
    for (int64_t f = 0; f < nf; ++f) {
        uvtri t;
        load_uvtri(uv, f, W, H, &t);
        int32_t i0 = F[3 * f], i1 = F[3 * f + 1], i2 = F[3 * f + 2];
        d3 v0 = ldf(V, i0), v1 = ldf(V, i1), v2 = ldf(V, i2);
        d3 e1 = sub(v1, v0), e2 = sub(v2, v0);
        double du1 = (double)(t.X[1] - t.X[0]), dv1 = (double)(t.Y[1] - t.Y[0]);
        double du2 = (double)(t.X[2] - t.X[0]), dv2 = (double)(t.Y[2] - t.Y[0]);
        int bad = (t.a2 <= 13 && t.a2 >= -13);
        d3 Tf = mk(0, 0, 0), Bf = mk(0, 0, 0);
        if (!bad) {
            double det = (double)t.a2;
            Tf = scl(sub(scl(e1, dv2), scl(e2, dv1)), 1.0 / det);
            Bf = scl(sub(scl(e2, du1), scl(e1, du2)), 1.0 / det);
        }
        int32_t ids[3] = {i0, i1, i2};
        for (int k = 0; k < 3; ++k) {
            d3 n = ldd(N, ids[k]);
            d3 tk = bad ? mk(0, 0, 0) : sub(Tf, scl(n, dot(Tf, n)));
            if (bad || norm(tk) == 0.0) { tk = onb_tangent(n); if (!bad) bad = 2; }
            std3(T, 3 * f + k, normalize(tk));
        }
        double hs = dot(cross(ldd(N, i0), Tf), Bf);
        wsign[f] = hs < 0.0 ? -1.0 : 1.0;
        degen[f] = (uint8_t)(bad != 0);
    }
}

/* ------------------------------------------------- 4. closest hit (Sec. 6.4)
 * The paper locates a high-poly correspondence per texel and keeps hits within
 * a distance filter.  Reading: the closest intersection of the line
 * p + t d (both directions) with any high-poly triangle, |t| <= tmax
 * inclusive, no back-face culling; ties: equal |t| prefers t >= 0, equal t
 * prefers the lower triangle id.  The intersection is the watertight test of
 * Woop, Benthin and Wald (2013) in double precision, with a zero edge
 * function counted as inside. */
typedef struct { int kx, ky, kz; double Sx, Sy, Sz; d3 o; } ray_t;

static ray_t make_ray(d3 o, d3 d) {
    ray_t r;
    double ax = fabs(d.x), ay = fabs(d.y), az = fabs(d.z);
    r.kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    r.kx = (r.kz + 1) % 3;
    r.ky = (r.kx + 1) % 3;
    if (comp(d, r.kz) < 0.0) { int tmp = r.kx; r.kx = r.ky; r.ky = tmp; }
    r.Sx = comp(d, r.kx) / comp(d, r.kz);
    r.Sy = comp(d, r.ky) / comp(d, r.kz);
    r.Sz = 1.0 / comp(d, r.kz);
    r.o = o;
    return r;
}

typedef struct { int tri; double t, b[3]; } hit_t;

static int isect(const ray_t *r, d3 A, d3 B, d3 C, double *t, double b[3]) {
    d3 a = sub(A, r->o), bb = sub(B, r->o), c = sub(C, r->o);
    double Ax = comp(a, r->kx) - r->Sx * comp(a, r->kz), Ay = comp(a, r->ky) - r->Sy * comp(a, r->kz);
    double Bx = comp(bb, r->kx) - r->Sx * comp(bb, r->kz), By = comp(bb, r->ky) - r->Sy * comp(bb, r->kz);
    double Cx = comp(c, r->kx) - r->Sx * comp(c, r->kz), Cy = comp(c, r->ky) - r->Sy * comp(c, r->kz);
    double U = Cx * By - Cy * Bx;
    double Vv = Ax * Cy - Ay * Cx;
    double W = Bx * Ay - By * Ax;
    if ((U < 0.0 || Vv < 0.0 || W < 0.0) && (U > 0.0 || Vv > 0.0 || W > 0.0)) return 0;
    double det = U + Vv + W;
    if (det == 0.0) return 0;
    double Az = r->Sz * comp(a, r->kz), Bz = r->Sz * comp(bb, r->kz), Cz = r->Sz * comp(c, r->kz);
    double T = U * Az + Vv * Bz + W * Cz;
    *t = T / det;
    b[0] = U / det; b[1] = Vv / det; b[2] = W / det;
    return 1;
}

/* the same edge functions without the inside test: the line's parameter and
 * signed barycentrics on the plane of (A, B, C); 0 when the line is parallel */
static int plane_hit(const ray_t *r, d3 A, d3 B, d3 C, double *t, double b[3]) {
    d3 a = sub(A, r->o), bb = sub(B, r->o), c = sub(C, r->o);
    double Ax = comp(a, r->kx) - r->Sx * comp(a, r->kz), Ay = comp(a, r->ky) - r->Sy * comp(a, r->kz);
    double Bx = comp(bb, r->kx) - r->Sx * comp(bb, r->kz), By = comp(bb, r->ky) - r->Sy * comp(bb, r->kz);
    double Cx = comp(c, r->kx) - r->Sx * comp(c, r->kz), Cy = comp(c, r->ky) - r->Sy * comp(c, r->kz);
    double U = Cx * By - Cy * Bx, Vv = Ax * Cy - Ay * Cx, W = Bx * Ay - By * Ax;
    double det = U + Vv + W;
    if (det == 0.0) return 0;
    double T = U * r->Sz * comp(a, r->kz) + Vv * r->Sz * comp(bb, r->kz) + W * r->Sz * comp(c, r->kz);
    *t = T / det;
    b[0] = U / det; b[1] = Vv / det; b[2] = W / det;
    return 1;
}

static int better(double t, int id, const hit_t *best) {
    if (best->tri < 0) return 1;
    double at = fabs(t), ab = fabs(best->t);
    if (at != ab) return at < ab;
    if ((t >= 0.0) != (best->t >= 0.0)) return t >= 0.0;
    return id < best->tri;
}

static int shares_vertex(const int32_t *F, int a, int b) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (F[3 * a + i] == F[3 * b + j]) return 1;
    return 0;
}

static void test_tri(const float *V, const int32_t *F, int tri, const ray_t *r, double tmax, int exclude, hit_t *best) {
    if (exclude >= 0 && shares_vertex(F, tri, exclude)) return;
    double t, b[3];
    if (!isect(r, ldf(V, F[3 * tri]), ldf(V, F[3 * tri + 1]), ldf(V, F[3 * tri + 2]), &t, b)) return;
    if (fabs(t) > tmax) return;
    if (better(t, tri, best)) { best->tri = tri; best->t = t; best->b[0] = b[0]; best->b[1] = b[1]; best->b[2] = b[2]; }
}

/* --- median-split BVH (binary, FP64 exact vertex bounds, leaves <= 4) */
typedef struct { double lo[3], hi[3]; int left, right, first, count; } bnode;
typedef struct { bnode *nodes; int nn; int *idx; const float *V; const int32_t *F; int64_t nf; } obvh;

static int cmp_axis;
static const double *cmp_cent;
static int cent_cmp(const void *a, const void *b) {
    double x = cmp_cent[3 * *(const int *)a + cmp_axis], y = cmp_cent[3 * *(const int *)b + cmp_axis];
    if (x < y) return -1;
    if (x > y) return 1;
    return *(const int *)a - *(const int *)b;
}

static int bvh_rec(obvh *b, double *cent, int first, int count) {
    int id = b->nn++;
    bnode *n = &b->nodes[id];
    for (int k = 0; k < 3; ++k) { n->lo[k] = INFINITY; n->hi[k] = -INFINITY; }
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = first; i < first + count; ++i) {
        int tr = b->idx[i];
        for (int v = 0; v < 3; ++v) {
            d3 p = ldf(b->V, b->F[3 * tr + v]);
            for (int k = 0; k < 3; ++k) {
                double c = comp(p, k);
                if (c < n->lo[k]) n->lo[k] = c;
                if (c > n->hi[k]) n->hi[k] = c;
            }
        }
        for (int k = 0; k < 3; ++k) {
            double c = cent[3 * tr + k];
            if (c < clo[k]) clo[k] = c;
            if (c > chi[k]) chi[k] = c;
        }
    }
    if (count <= 4) { n->left = n->right = -1; n->first = first; n->count = count; return id; }
    int ax = 0;
    for (int k = 1; k < 3; ++k) if (chi[k] - clo[k] > chi[ax] - clo[ax]) ax = k;
    cmp_axis = ax; cmp_cent = cent;
    qsort(b->idx + first, (size_t)count, sizeof(int), cent_cmp);
    int half = count / 2;
    int l = bvh_rec(b, cent, first, half);
    int r = bvh_rec(b, cent, first + half, count - half);
    n = &b->nodes[id];
    n->left = l; n->right = r; n->first = first; n->count = 0;
    return id;
}

void *or_bvh_build(const float *V, const int32_t *F, int64_t nf) {
    obvh *b = (obvh *)calloc(1, sizeof(obvh));
    if (!b) return NULL;
    b->V = V; b->F = F; b->nf = nf;
    b->nodes = (bnode *)malloc(sizeof(bnode) * (size_t)(2 * nf + 1));
    b->idx = (int *)malloc(sizeof(int) * (size_t)(nf > 0 ? nf : 1));
    double *cent = (double *)malloc(sizeof(double) * 3 * (size_t)(nf > 0 ? nf : 1));
    if (!b->nodes || !b->idx || !cent) { free(b->nodes); free(b->idx); free(cent); free(b); return NULL; }
    for (int64_t i = 0; i < nf; ++i) {
        b->idx[i] = (int)i;
        d3 c = scl(add(add(ldf(V, F[3 * i]), ldf(V, F[3 * i + 1])), ldf(V, F[3 * i + 2])), 1.0 / 3.0);
        std3(cent, i, c);
    }
    if (nf > 0) bvh_rec(b, cent, 0, (int)nf);
    free(cent);
    return b;
}

void or_bvh_free(void *p) {
    obvh *b = (obvh *)p;
    if (!b) return;
    free(b->nodes); free(b->idx); free(b);
}

/* parameter interval of the line o + t d inside the box, widened so that
 * rounding can only enlarge it; returns 0 when the line misses the box */
static int box_interval(const bnode *n, d3 o, d3 d, double *t0, double *t1) {
    double lo = -INFINITY, hi = INFINITY;
    for (int k = 0; k < 3; ++k) {
        double ok = comp(o, k), dk = comp(d, k);
        if (dk == 0.0) {
            if (ok < n->lo[k] || ok > n->hi[k]) return 0;
            continue;
        }
        double a = (n->lo[k] - ok) / dk, b = (n->hi[k] - ok) / dk;
        if (a > b) { double tmp = a; a = b; b = tmp; }
        if (a > lo) lo = a;
        if (b < hi) hi = b;
    }
    double eps = 1e-9 * (fabs(lo) + fabs(hi)) + 1e-12;
    *t0 = lo - eps; *t1 = hi + eps;
    return *t0 <= *t1;
}

static void bvh_closest(const obvh *b, const ray_t *r, d3 o, d3 d, double tmax, int exclude, hit_t *best) {
    if (b->nf == 0) return;
    int stack[256], sp = 0;
    stack[sp++] = 0;
    while (sp) {
        const bnode *n = &b->nodes[stack[--sp]];
        double t0, t1;
        if (!box_interval(n, o, d, &t0, &t1)) continue;
        double lim = best->tri >= 0 ? fabs(best->t) : tmax;
        if (t0 > lim || t1 < -lim) continue;
        if (n->left < 0) {
            for (int i = n->first; i < n->first + n->count; ++i) test_tri(b->V, b->F, b->idx[i], r, tmax, exclude, best);
        } else {
            stack[sp++] = n->left;
            stack[sp++] = n->right;
        }
    }
}

static void closest(const float *V, const int32_t *F, int64_t nf, const obvh *bvh, d3 o, d3 d, double tmax, int exclude, hit_t *best) {
    ray_t r = make_ray(o, d);
    best->tri = -1; best->t = 0.0; best->b[0] = best->b[1] = best->b[2] = 0.0;
    if (bvh) { bvh_closest(bvh, &r, o, d, tmax, exclude, best); return; }
    for (int64_t i = 0; i < nf; ++i) test_tri(V, F, (int)i, &r, tmax, exclude, best);
}

/* exposed for pin tests: out = {tri, t, b0, b1, b2} */
int or_closest_hit(const float *V, const int32_t *F, int64_t nf, void *bvh, const double *o, const double *d, double tmax, double *out) {
    hit_t h;
    closest(V, F, nf, (const obvh *)bvh, mk(o[0], o[1], o[2]), mk(d[0], d[1], d[2]), tmax, -1, &h);
    out[0] = h.tri; out[1] = h.t; out[2] = h.b[0]; out[3] = h.b[1]; out[4] = h.b[2];
    return h.tri >= 0;
}

/* ------------------------------------------------- 4b. closest-point query
 * The correspondence as Sec. 6.4 words it: for the texel's world-space
 * position, the nearest point of the high-poly surface.  Definition used:
 * over every high-poly triangle (a closed set) the point x minimising
 * |x - p|.  A triangle's own closest point is the foot of the perpendicular
 * from p when the foot lies in the closed triangle, else the nearest of the
 * clamped projections of p onto its three edges (a zero-area triangle has
 * only its edges).  Equal distances prefer the lower triangle id.  The
 * distance filter of Sec. 6.4 keeps |x - p| <= max_dist (inclusive). */
typedef struct { int tri; double d2; d3 x; double b[3]; } cpt_t;

static double tri_closest(d3 p, d3 A, d3 B, d3 C, d3 *x, double b[3]) {
    d3 n = cross(sub(B, A), sub(C, A));
    double nn = dot(n, n);
    if (nn > 0.0) {
        double h = dot(sub(p, A), n);
        d3 f = sub(p, scl(n, h / nn));
        double ba = dot(cross(sub(C, B), sub(f, B)), n) / nn;
        double bb = dot(cross(sub(A, C), sub(f, C)), n) / nn;
        double bc = dot(cross(sub(B, A), sub(f, A)), n) / nn;
        if (ba >= 0.0 && bb >= 0.0 && bc >= 0.0) {
            *x = f;
            b[0] = ba; b[1] = bb; b[2] = bc;
            return h * h / nn;
        }
    }
    const d3 P[3] = {A, B, C};
    double best = INFINITY;
    for (int k = 0; k < 3; ++k) {
        d3 a = P[k], e = sub(P[(k + 1) % 3], a);
        double ee = dot(e, e), s = ee > 0.0 ? dot(sub(p, a), e) / ee : 0.0;
        if (s < 0.0) s = 0.0;
        if (s > 1.0) s = 1.0;
        d3 y = add(a, scl(e, s));
        d3 w = sub(p, y);
        double d2 = dot(w, w);
        if (d2 < best) {
            best = d2;
            *x = y;
            b[k] = 1.0 - s; b[(k + 1) % 3] = s; b[(k + 2) % 3] = 0.0;
        }
    }
    return best;
}

static void cp_test(const float *V, const int32_t *F, int tri, d3 p, double r2, cpt_t *best) {
    d3 x;
    double b[3];
    double d2 = tri_closest(p, ldf(V, F[3 * tri]), ldf(V, F[3 * tri + 1]), ldf(V, F[3 * tri + 2]), &x, b);
    if (d2 > r2) return;
    if (best->tri >= 0 && (d2 > best->d2 || (d2 == best->d2 && tri > best->tri))) return;
    best->tri = tri; best->d2 = d2; best->x = x;
    best->b[0] = b[0]; best->b[1] = b[1]; best->b[2] = b[2];
}

static double box_d2(const bnode *n, d3 p) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
        double c = comp(p, k), e = 0.0;
        if (c < n->lo[k]) e = n->lo[k] - c;
        else if (c > n->hi[k]) e = c - n->hi[k];
        s += e * e;
    }
    return s;
}

/* a box is skipped only when it lies farther than the bound plus a relative
 * 1e-9 and an absolute 1e-24, which covers every rounding of the box and
 * triangle distances: the result is bit for bit that of brute force */
static int box_beyond(double bd2, double lim) { return bd2 > lim * (1.0 + 1e-9) + 1e-24; }

static void bvh_cp(const obvh *b, d3 p, double r2, cpt_t *best) {
    if (b->nf == 0) return;
    int stack[256], sp = 0;
    stack[sp++] = 0;
    while (sp) {
        const bnode *n = &b->nodes[stack[--sp]];
        if (box_beyond(box_d2(n, p), best->tri >= 0 ? best->d2 : r2)) continue;
        if (n->left < 0) {
            for (int i = n->first; i < n->first + n->count; ++i) cp_test(b->V, b->F, b->idx[i], p, r2, best);
        } else {
            /* nearer child last, so it is popped first */
            double dl = box_d2(&b->nodes[n->left], p), dr = box_d2(&b->nodes[n->right], p);
            stack[sp++] = dl <= dr ? n->right : n->left;
            stack[sp++] = dl <= dr ? n->left : n->right;
        }
    }
}

static void closest_point(const float *V, const int32_t *F, int64_t nf, const obvh *bvh, d3 p, double rmax, cpt_t *best) {
    best->tri = -1; best->d2 = 0.0; best->x = p; best->b[0] = best->b[1] = best->b[2] = 0.0;
    double r2 = rmax * rmax;
    if (bvh) { bvh_cp(bvh, p, r2, best); return; }
    for (int64_t i = 0; i < nf; ++i) cp_test(V, F, (int)i, p, r2, best);
}

/* every triangle whose closest point lies within distance r of p */
typedef void (*cp_visit_fn)(void *ctx, int tri, d3 x, const double b[3]);
static void cp_range(const float *V, const int32_t *F, int64_t nf, const obvh *bvh, d3 p, double r, cp_visit_fn fn, void *ctx) {
    double r2 = r * r;
    if (!bvh) {
        for (int64_t i = 0; i < nf; ++i) {
            d3 x; double b[3];
            if (tri_closest(p, ldf(V, F[3 * i]), ldf(V, F[3 * i + 1]), ldf(V, F[3 * i + 2]), &x, b) <= r2) fn(ctx, (int)i, x, b);
        }
        return;
    }
    if (bvh->nf == 0) return;
    int stack[256], sp = 0;
    stack[sp++] = 0;
    while (sp) {
        const bnode *n = &bvh->nodes[stack[--sp]];
        if (box_beyond(box_d2(n, p), r2)) continue;
        if (n->left < 0) {
            for (int i = n->first; i < n->first + n->count; ++i) {
                int t = bvh->idx[i];
                d3 x; double b[3];
                if (tri_closest(p, ldf(V, F[3 * t]), ldf(V, F[3 * t + 1]), ldf(V, F[3 * t + 2]), &x, b) <= r2) fn(ctx, t, x, b);
            }
        } else {
            stack[sp++] = n->left;
            stack[sp++] = n->right;
        }
    }
}

/* exposed for pin tests: out = {tri, d2, x[3], b[3]} */
int or_closest_point(const float *V, const int32_t *F, int64_t nf, void *bvh, const double *p, double rmax, double *out) {
    cpt_t c;
    closest_point(V, F, nf, (const obvh *)bvh, mk(p[0], p[1], p[2]), rmax, &c);
    out[0] = c.tri; out[1] = c.d2;
    out[2] = c.x.x; out[3] = c.x.y; out[4] = c.x.z;
    out[5] = c.b[0]; out[6] = c.b[1]; out[7] = c.b[2];
    return c.tri >= 0;
}

/* ------------------------------------------------- 4-5. trace + shade
 * Per ray texel (Sec. 6.4): the correspondence on the high surface within the
 * distance filter, its barycentric smooth normal, the projection into the
 * texel tangent frame.  Two correspondence queries:
 *   ray (query 0): the line from the texel's surface point p along its
 *     interpolated normal d, closest |t| <= max_dist, disp = t;
 *   closest point (query 1): the point x of the high surface nearest to p,
 *     |x - p| <= max_dist, disp = |x - p| signed by (x - p) . d (>= 0 is +).
 * Readings: misses and unreliable (degenerate-UV) texels get (0,0,1);
 * disp = 0 on a miss.
 * Exception flags (texels where several results are equally correct):
 *   bit0 ray: hit with min barycentric < 1e-5 (near a high-poly edge)
 *   bit1 closest |t| or distance within 1e-5*diam of max_dist
 *   bit2 texel centre within 1e-5 texel of an edge of its low face
 *   bit3 ray: a triangle sharing no vertex with the hit lies within
 *        1e-5*diam in |t|; closest point: another triangle within 1e-7*diam
 *        of the distance gives a hit normal more than 1e-5 away or, at a
 *        distance above 5e-7*diam, the other displacement sign; or there
 *        (x - p) . d is within 1e-7*diam of zero (the sign is a rounding
 *        decision).  Below 5e-7*diam either sign is within the tolerance.
 */
typedef struct {
    const float *hv; const int32_t *hf; int64_t nhf; const double *hn; const obvh *bvh;
    const float *lv; const int32_t *lf; const double *ln; const float *luv;
    const double *T; const double *wsign; const uint8_t *degen;
    const int32_t *face; const double *bary;
    int W, H; double max_dist, diam;
    const int64_t *texels; int64_t ntex;
    uint8_t *mask; double *nts; double *disp; int32_t *hit_tri; double *hit_t; double *hit_b; uint8_t *flags;
    int query;
    const int32_t *force;   /* optional [W*H]: evaluate this triangle instead of searching */
    int nthreads, tid;
} trace_job;

static double seg_dist_units(double cx, double cy, double ax, double ay, double bx, double by) {
    double dx = bx - ax, dy = by - ay, wx = cx - ax, wy = cy - ay;
    double dd = dx * dx + dy * dy, s = dd > 0 ? (wx * dx + wy * dy) / dd : 0.0;
    if (s < 0) s = 0;
    if (s > 1) s = 1;
    double px = ax + s * dx - cx, py = ay + s * dy - cy;
    return sqrt(px * px + py * py);
}

/* barycentric smooth normal of the high mesh on triangle tri */
static d3 hit_normal(const trace_job *j, int tri, const double b[3]) {
    d3 m = mk(0, 0, 0);
    for (int k = 0; k < 3; ++k) m = add(m, scl(ldd(j->hn, j->hf[3 * tri + k]), b[k]));
    return normalize(m);
}

/* the other triangles near the closest distance (flag bit3) */
typedef struct { const trace_job *j; int tri; d3 nh, p, d; int pos, sign_matters; int ambiguous; } cp_amb_t;

static void cp_amb_visit(void *ctx, int tri, d3 x, const double b[3]) {
    cp_amb_t *a = (cp_amb_t *)ctx;
    if (tri == a->tri || a->ambiguous) return;
    d3 nh = hit_normal(a->j, tri, b);
    d3 e = sub(nh, a->nh);
    double dev = fmax(fabs(e.x), fmax(fabs(e.y), fabs(e.z)));
    int pos = dot(sub(x, a->p), a->d) >= 0.0;
    if (dev > 1e-5 || (a->sign_matters && pos != a->pos)) a->ambiguous = 1;
}

static void trace_one(const trace_job *j, int64_t tex) {
    int32_t f = j->face[tex];
    if (f < 0) return;
    const double *b = j->bary + 3 * tex;
    int32_t ids[3] = {j->lf[3 * f], j->lf[3 * f + 1], j->lf[3 * f + 2]};
    d3 p = mk(0, 0, 0), s = mk(0, 0, 0), ts = mk(0, 0, 0);
    for (int k = 0; k < 3; ++k) {
        p = add(p, scl(ldf(j->lv, ids[k]), b[k]));
        s = add(s, scl(ldd(j->ln, ids[k]), b[k]));
        ts = add(ts, scl(ldd(j->T, 3 * f + k), b[k]));
    }
    d3 d = normalize(s);
    double tol = 1e-5 * j->diam;
    uint8_t fl = 0;
    int hit = 0, tri = -1;
    double disp = 0.0, hb[3] = {0.0, 0.0, 0.0};
    if (j->force) {
        /* The given triangle alone, for checking an answer of another
         * implementation where several are equally correct: the ray query
         * takes the line's crossing of its plane (signed barycentrics, so a
         * triangle missed by a hair shows a slightly negative one), the
         * closest-point query its nearest point.  No filter, no flags. */
        tri = j->force[tex];
        if (tri < 0) return;
        d3 A = ldf(j->hv, j->hf[3 * tri]), B = ldf(j->hv, j->hf[3 * tri + 1]), C = ldf(j->hv, j->hf[3 * tri + 2]);
        if (j->query == 0) {
            ray_t r = make_ray(p, d);
            hit = plane_hit(&r, A, B, C, &disp, hb);
        } else {
            d3 x;
            double dist = sqrt(tri_closest(p, A, B, C, &x, hb));
            disp = dot(sub(x, p), d) >= 0.0 ? dist : -dist;
            hit = 1;
        }
        if (!hit) { tri = -1; disp = 0.0; }
    } else if (j->query == 0) {
        hit_t h;
        closest(j->hv, j->hf, j->nhf, j->bvh, p, d, j->max_dist + tol, -1, &h);
        hit = h.tri >= 0 && fabs(h.t) <= j->max_dist;
        if (h.tri >= 0 && fabs(h.t) >= j->max_dist - tol) fl |= 2;
        if (hit) {
            double mb = h.b[0] < h.b[1] ? h.b[0] : h.b[1];
            if (h.b[2] < mb) mb = h.b[2];
            if (mb < 1e-5) fl |= 1;
            hit_t h2;
            closest(j->hv, j->hf, j->nhf, j->bvh, p, d, fabs(h.t) + tol, h.tri, &h2);
            if (h2.tri >= 0) fl |= 8;
        }
        tri = h.tri;
        disp = h.tri >= 0 ? h.t : 0.0;
        for (int k = 0; k < 3; ++k) hb[k] = h.tri >= 0 ? h.b[k] : 0.0;
    } else {
        cpt_t c;
        closest_point(j->hv, j->hf, j->nhf, j->bvh, p, j->max_dist + tol, &c);
        double dist = sqrt(c.d2);
        hit = c.tri >= 0 && dist <= j->max_dist;
        if (c.tri >= 0 && dist >= j->max_dist - tol) fl |= 2;
        if (c.tri >= 0) {
            double along = dot(sub(c.x, p), d);
            double tolc = 1e-7 * j->diam;
            int sign_matters = dist > 5.0 * tolc;
            cp_amb_t a = {j, c.tri, hit_normal(j, c.tri, c.b), p, d, along >= 0.0, sign_matters, 0};
            cp_range(j->hv, j->hf, j->nhf, j->bvh, p, dist + tolc, cp_amb_visit, &a);
            if (a.ambiguous || (sign_matters && fabs(along) <= tolc)) fl |= 8;
            disp = along >= 0.0 ? dist : -dist;
        }
        tri = c.tri;
        for (int k = 0; k < 3; ++k) hb[k] = c.b[k];
    }
    {
        int x = (int)(tex % j->W), y = (int)(tex / j->W);
        double cx = 256.0 * x + 128.0, cy = 256.0 * y + 128.0;
        double X[3], Y[3];
        for (int k = 0; k < 3; ++k) {
            X[k] = (double)or_snap(j->luv[6 * f + 2 * k], j->W);
            Y[k] = (double)or_snap(j->luv[6 * f + 2 * k + 1], j->H);
        }
        for (int k = 0; k < 3; ++k)
            if (seg_dist_units(cx, cy, X[k], Y[k], X[(k + 1) % 3], Y[(k + 1) % 3]) < 1e-5 * 256.0) fl |= 4;
    }
    d3 n_ts = mk(0, 0, 1);
    if (hit && !j->degen[f]) {
        d3 N = d;
        d3 Tt = normalize(sub(ts, scl(N, dot(ts, N))));
        d3 B = scl(cross(N, Tt), j->wsign[f]);
        d3 nh = hit_normal(j, tri, hb);
        n_ts = mk(dot(nh, Tt), dot(nh, B), dot(nh, N));
    }
    j->mask[tex] = (uint8_t)hit;
    std3(j->nts, tex, n_ts);
    j->disp[tex] = hit ? disp : 0.0;
    j->hit_tri[tex] = hit ? tri : -1;
    j->hit_t[tex] = tri >= 0 ? disp : 0.0;
    for (int k = 0; k < 3; ++k) j->hit_b[3 * tex + k] = tri >= 0 ? hb[k] : 0.0;
    j->flags[tex] = fl;
}

static void *trace_worker(void *arg) {
    trace_job *j = (trace_job *)arg;
    for (int64_t i = j->tid; i < j->ntex; i += j->nthreads) trace_one(j, j->texels ? j->texels[i] : i);
    return NULL;
}

int or_trace(const float *hv, int64_t nhv, const int32_t *hf, int64_t nhf, const double *hn, void *bvh,
             const float *lv, const int32_t *lf, const double *ln, const float *luv,
             const double *T, const double *wsign, const uint8_t *degen,
             const int32_t *face, const double *bary, int W, int H, double max_dist, double diam,
             const int64_t *texels, int64_t ntex, int nthreads,
             uint8_t *mask, double *nts, double *disp, int32_t *hit_tri, double *hit_t, double *hit_b, uint8_t *flags,
             int query, const int32_t *force) {
    (void)nhv;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    trace_job base = {hv, hf, nhf, hn, (const obvh *)bvh, lv, lf, ln, luv, T, wsign, degen, face, bary,
                      W, H, max_dist, diam, texels, texels ? ntex : (int64_t)W * H,
                      mask, nts, disp, hit_tri, hit_t, hit_b, flags, query, force, nthreads, 0};
    trace_job jobs[256];
    pthread_t th[256];
    for (int i = 0; i < nthreads; ++i) { jobs[i] = base; jobs[i].tid = i; }
    for (int i = 1; i < nthreads; ++i)
        if (pthread_create(&th[i], NULL, trace_worker, &jobs[i])) return -1;
    trace_worker(&jobs[0]);
    for (int i = 1; i < nthreads; ++i) pthread_join(th[i], NULL);
    return 0;
}

/* ------------------------------------------------- "baked mean" (Sec. 6.1)
 * The quality measure of a baked normal map that the simplification benchmark
 * reports: at points spread uniformly by area over the simplified (low) mesh,
 * the angle between the normal the map gives there and the true normal of
 * the raw (high) mesh, averaged over the points.  Readings of what the paper
 * leaves open:
 *  - sample k is given by the caller: face f_k and barycentrics
 *    (1 - b1 - b2, b1, b2);
 *  - the map is read at the texel holding the sample's UV point,
 *    x = floor(u W), y = floor(v H) (clamped to the atlas), unfiltered; the
 *    RGB codes decode as c = (q - 128) / 127 (the inverse of the encoding of
 *    section 6) and the vector is renormalised;
 *  - it is taken to world space through the tangent frame of the bake at the
 *    sample point: N = normalize(sum b_i n_i), T = the interpolated corner
 *    tangents made orthogonal to N, B = w (N x T); on a face the
 *    UV-reliability filter marks (degenerate UVs, whose frame is bookkeeping
 *    only) the map is not used and the normal is N, as a neutral texel gives;
 *  - the raw mesh's true normal is its area-weighted smooth normal,
 *    interpolated at the point of the raw surface nearest to the sample
 *    (within max_dist; with none, the angle is -1);
 *  - angle = atan2(|a x b|, a . b), in degrees.
 * flags bit0: another raw triangle within 1e-7 * diam of the nearest distance
 * gives a smooth normal more than 1e-5 away (two correct answers). */
typedef struct {
    trace_job j;
    const int32_t *sface; const double *sbary; int64_t n;
    const uint8_t *rgba; double *angle; uint8_t *sflags;
} map_err_job;

static void map_error_one(const map_err_job *m, int64_t k) {
    const trace_job *j = &m->j;
    int32_t f = m->sface[k];
    double b[3] = {1.0 - m->sbary[2 * k] - m->sbary[2 * k + 1], m->sbary[2 * k], m->sbary[2 * k + 1]};
    int32_t ids[3] = {j->lf[3 * f], j->lf[3 * f + 1], j->lf[3 * f + 2]};
    d3 p = mk(0, 0, 0), s = mk(0, 0, 0), ts = mk(0, 0, 0);
    double u = 0.0, v = 0.0;
    for (int q = 0; q < 3; ++q) {
        p = add(p, scl(ldf(j->lv, ids[q]), b[q]));
        s = add(s, scl(ldd(j->ln, ids[q]), b[q]));
        ts = add(ts, scl(ldd(j->T, 3 * f + q), b[q]));
        u += b[q] * j->luv[6 * f + 2 * q];
        v += b[q] * j->luv[6 * f + 2 * q + 1];
    }
    d3 N = normalize(s);
    d3 Tt = normalize(sub(ts, scl(N, dot(ts, N))));
    d3 B = scl(cross(N, Tt), j->wsign[f]);
    int x = (int)floor(u * j->W), y = (int)floor(v * j->H);
    if (x < 0) x = 0;
    if (x > j->W - 1) x = j->W - 1;
    if (y < 0) y = 0;
    if (y > j->H - 1) y = j->H - 1;
    const uint8_t *q8 = m->rgba + 4 * ((int64_t)y * j->W + x);
    d3 c = normalize(mk((q8[0] - 128.0) / 127.0, (q8[1] - 128.0) / 127.0, (q8[2] - 128.0) / 127.0));
    d3 nm = j->degen[f] ? N : normalize(add(add(scl(Tt, c.x), scl(B, c.y)), scl(N, c.z)));
    cpt_t cp;
    closest_point(j->hv, j->hf, j->nhf, j->bvh, p, j->max_dist, &cp);
    m->sflags[k] = 0;
    if (cp.tri < 0) { m->angle[k] = -1.0; return; }
    d3 nr = hit_normal(j, cp.tri, cp.b);
    m->angle[k] = atan2(norm(cross(nm, nr)), dot(nm, nr)) * (180.0 / 3.14159265358979323846);
    cp_amb_t a = {j, cp.tri, nr, p, N, 1, 0, 0};
    cp_range(j->hv, j->hf, j->nhf, j->bvh, p, sqrt(cp.d2) + 1e-7 * j->diam, cp_amb_visit, &a);
    if (a.ambiguous) m->sflags[k] |= 1;
}

static void *map_error_worker(void *arg) {
    map_err_job *m = (map_err_job *)arg;
    for (int64_t k = m->j.tid; k < m->n; k += m->j.nthreads) map_error_one(m, k);
    return NULL;
}

int or_normal_map_error(const float *hv, int64_t nhf_unused, const int32_t *hf, int64_t nhf, const double *hn,
                        void *bvh, const float *lv, const int32_t *lf, const double *ln, const float *luv,
                        const double *T, const double *wsign, const uint8_t *degen, int W, int H,
                        const uint8_t *rgba,
                        const int32_t *sface, const double *sbary, int64_t n, double max_dist, double diam,
                        int nthreads, double *angle, uint8_t *sflags) {
    (void)nhf_unused;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    map_err_job base;
    memset(&base, 0, sizeof(base));
    base.j.hv = hv; base.j.hf = hf; base.j.nhf = nhf; base.j.hn = hn; base.j.bvh = (const obvh *)bvh;
    base.j.lv = lv; base.j.lf = lf; base.j.ln = ln; base.j.luv = luv; base.j.T = T; base.j.wsign = wsign;
    base.j.degen = degen;
    base.j.W = W; base.j.H = H; base.j.max_dist = max_dist; base.j.diam = diam; base.j.nthreads = nthreads;
    base.sface = sface; base.sbary = sbary; base.n = n; base.rgba = rgba; base.angle = angle; base.sflags = sflags;
    map_err_job jobs[256];
    pthread_t th[256];
    for (int i = 0; i < nthreads; ++i) { jobs[i] = base; jobs[i].j.tid = i; }
    for (int i = 1; i < nthreads; ++i)
        if (pthread_create(&th[i], NULL, map_error_worker, &jobs[i])) return -1;
    map_error_worker(&jobs[0]);
    for (int i = 1; i < nthreads; ++i) pthread_join(th[i], NULL);
    return 0;
}

/* ------------------------------------------------- 6. encode + dilation
 * RGB8 encoding (Sec. 6.4), reading: q = 128 + round_half_away(127*c)
 * for c clamped to [-1, 1] (codes 1..255, 128 = 0).  The unsigned mapping
 * floor((c/2 + 1/2)*255 + 1/2) would put the 127/128 code boundary exactly at
 * c = 0, the value every texel takes where the high surface runs parallel to
 * the low one, leaving that code to rounding noise; here 0 sits in the middle
 * of code 128.  A = 255 on ray and dilated texels, else 0; untouched texels
 * encode (0,0,1) = (128,128,255).
 * Dilation across UV seams (Sec. 6.4), reading: `gutter` passes; each
 * pass gives every unfilled texel with at least one filled 8-neighbour (as of
 * the previous pass) the renormalised mean of those neighbours' tangent-space
 * normals and the mean of their displacements.  The hit mask is not dilated. */
/* The code is taken from the FP64 component itself; a kernel working in a
 * narrower precision may land one code away where 127*c lies within its
 * rounding of a half-integer, which the comparison's 1-LSB allowance covers. */
static uint8_t enc(double c) {
    double v = c;
    if (v < -1.0) v = -1.0;
    if (v > 1.0) v = 1.0;
    double r = v * 127.0;
    double q = r >= 0.0 ? floor(r + 0.5) : -floor(-r + 0.5);
    return (uint8_t)(128 + (int)q);
}

void or_encode(const double *nts, const uint8_t *filled, int64_t n, uint8_t *rgba) {
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) rgba[4 * i + k] = enc(nts[3 * i + k]);
        rgba[4 * i + 3] = filled[i] ? 255 : 0;
    }
}

/* filled: 1 for ray texels on input; dilated texels get 2.  Untouched texels
 * get nts = (0,0,1), disp = 0. */
int or_dilate(int W, int H, int gutter, uint8_t *filled, double *nts, double *disp) {
    int64_t n = (int64_t)W * H;
    uint8_t *prev = (uint8_t *)malloc((size_t)n);
    if (!prev) return -1;
    for (int64_t i = 0; i < n; ++i)
        if (!filled[i]) { nts[3 * i] = 0; nts[3 * i + 1] = 0; nts[3 * i + 2] = 1; disp[i] = 0; }
    for (int pass = 0; pass < gutter; ++pass) {
        memcpy(prev, filled, (size_t)n);
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                int64_t i = (int64_t)y * W + x;
                if (prev[i]) continue;
                d3 m = mk(0, 0, 0);
                double dsum = 0.0;
                int cnt = 0;
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int xx = x + dx, yy = y + dy;
                        if ((dx == 0 && dy == 0) || xx < 0 || yy < 0 || xx >= W || yy >= H) continue;
                        int64_t q = (int64_t)yy * W + xx;
                        if (!prev[q]) continue;
                        m = add(m, ldd(nts, q));
                        dsum += disp[q];
                        ++cnt;
                    }
                if (!cnt) continue;
                d3 mm = scl(m, 1.0 / cnt);
                std3(nts, i, norm(mm) > 0 ? normalize(mm) : mk(0, 0, 1));
                disp[i] = dsum / cnt;
                filled[i] = 2;
            }
    }
    free(prev);
    return 0;
}

/* ------------------------------------------------- 7. loss + analytic gradient
 * L = (1/|M|) sum_{k in M} t_k^2 + lambda (1/|M|) sum_{k in M} (1 - n_hit,k . d_k)
 * over the hit texels M, the hit triangle of each texel held fixed; t is the
 * intersection of the line with the hit triangle's plane and the hit
 * barycentrics those of the intersection point, so L is smooth in the low
 * positions.  grad [nlv*3] receives dL/dV_low (pass NULL for the loss only). */
double or_loss_grad(const float *hv, const int32_t *hf, const double *hn,
                    const double *lvd /* low positions in FP64 [nlv*3] */, int64_t nlv, const int32_t *lf, int64_t nlf,
                    const int32_t *face, const double *bary, const int32_t *hit_tri, int64_t ntex,
                    double lambda, double *grad) {
    /* vertex normals of the (possibly perturbed) low mesh, FP64 */
    double *acc = (double *)calloc((size_t)nlv * 3, sizeof(double));
    double *gn = grad ? (double *)calloc((size_t)nlv * 3, sizeof(double)) : NULL;
    for (int64_t f = 0; f < nlf; ++f) {
        d3 a = ldd(lvd, lf[3 * f]), b = ldd(lvd, lf[3 * f + 1]), c = ldd(lvd, lf[3 * f + 2]);
        d3 cr = cross(sub(b, a), sub(c, a));
        for (int k = 0; k < 3; ++k) std3(acc, lf[3 * f + k], add(ldd(acc, lf[3 * f + k]), cr));
    }
    if (grad) memset(grad, 0, sizeof(double) * 3 * (size_t)nlv);
    int64_t count = 0;
    double sum_t = 0.0, sum_n = 0.0;
    for (int64_t k = 0; k < ntex; ++k) if (face[k] >= 0 && hit_tri[k] >= 0) ++count;
    if (count == 0) { free(acc); free(gn); return 0.0; }
    double inv = 1.0 / (double)count;
    for (int64_t k = 0; k < ntex; ++k) {
        if (face[k] < 0 || hit_tri[k] < 0) continue;
        int32_t f = face[k];
        const double *b = bary + 3 * k;
        int32_t ids[3] = {lf[3 * f], lf[3 * f + 1], lf[3 * f + 2]};
        d3 p = mk(0, 0, 0), s = mk(0, 0, 0);
        d3 nv[3];
        for (int q = 0; q < 3; ++q) {
            nv[q] = normalize(ldd(acc, ids[q]));
            p = add(p, scl(ldd(lvd, ids[q]), b[q]));
            s = add(s, scl(nv[q], b[q]));
        }
        double sl = norm(s);
        d3 d = scl(s, 1.0 / sl);
        int h = hit_tri[k];
        d3 A = ldf(hv, hf[3 * h]), B = ldf(hv, hf[3 * h + 1]), C = ldf(hv, hf[3 * h + 2]);
        d3 Nh = cross(sub(B, A), sub(C, A));
        double nn = dot(Nh, Nh), dn = dot(d, Nh);
        double t = dot(sub(A, p), Nh) / dn;
        d3 x = add(p, scl(d, t));
        double beta[3] = {dot(cross(sub(C, B), sub(x, B)), Nh) / nn,
                          dot(cross(sub(A, C), sub(x, C)), Nh) / nn,
                          dot(cross(sub(B, A), sub(x, A)), Nh) / nn};
        d3 Nj[3] = {ldd(hn, hf[3 * h]), ldd(hn, hf[3 * h + 1]), ldd(hn, hf[3 * h + 2])};
        d3 m = add(add(scl(Nj[0], beta[0]), scl(Nj[1], beta[1])), scl(Nj[2], beta[2]));
        double ml = norm(m);
        d3 nh = scl(m, 1.0 / ml);
        sum_t += t * t;
        sum_n += 1.0 - dot(nh, d);
        if (!grad) continue;
        /* adjoint, unscaled by 1/|M| until the end */
        double gt = 2.0 * t;
        d3 g_nh = scl(d, -lambda);
        d3 g_d = scl(nh, -lambda);
        d3 g_m = scl(sub(g_nh, scl(nh, dot(nh, g_nh))), 1.0 / ml);
        double g_beta[3] = {dot(Nj[0], g_m), dot(Nj[1], g_m), dot(Nj[2], g_m)};
        d3 gradb[3] = {scl(cross(Nh, sub(C, B)), 1.0 / nn), scl(cross(Nh, sub(A, C)), 1.0 / nn), scl(cross(Nh, sub(B, A)), 1.0 / nn)};
        d3 g_x = add(add(scl(gradb[0], g_beta[0]), scl(gradb[1], g_beta[1])), scl(gradb[2], g_beta[2]));
        double g_tt = gt + dot(g_x, d);
        d3 g_p = sub(g_x, scl(Nh, g_tt / dn));
        g_d = add(g_d, scl(g_p, t));
        d3 g_s = scl(sub(g_d, scl(d, dot(d, g_d))), 1.0 / sl);
        for (int q = 0; q < 3; ++q) {
            std3(grad, ids[q], add(ldd(grad, ids[q]), scl(g_p, b[q])));
            std3(gn, ids[q], add(ldd(gn, ids[q]), scl(g_s, b[q])));
        }
    }
    if (grad) {
        /* through n_i = normalize(a_i), a_i = sum of face cross products */
        double *ga = (double *)calloc((size_t)nlv * 3, sizeof(double));
        for (int64_t i = 0; i < nlv; ++i) {
            d3 a = ldd(acc, i);
            double al = norm(a);
            if (al == 0.0) continue;
            d3 n = scl(a, 1.0 / al), g = ldd(gn, i);
            std3(ga, i, scl(sub(g, scl(n, dot(n, g))), 1.0 / al));
        }
        for (int64_t f = 0; f < nlf; ++f) {
            int32_t i0 = lf[3 * f], i1 = lf[3 * f + 1], i2 = lf[3 * f + 2];
            d3 g = add(add(ldd(ga, i0), ldd(ga, i1)), ldd(ga, i2));
            d3 e1 = sub(ldd(lvd, i1), ldd(lvd, i0)), e2 = sub(ldd(lvd, i2), ldd(lvd, i0));
            d3 g1 = cross(e2, g), g2 = cross(g, e1);
            std3(grad, i1, add(ldd(grad, i1), g1));
            std3(grad, i2, add(ldd(grad, i2), g2));
            std3(grad, i0, sub(ldd(grad, i0), add(g1, g2)));
        }
        for (int64_t i = 0; i < 3 * nlv; ++i) grad[i] *= inv;
        free(ga);
    }
    free(acc); free(gn);
    return (sum_t + lambda * sum_n) * inv;
}

/* ------------------------------------------------- 8. hidden-face removal (Sec. 6.2)
 * Visibility pass (the paper's viewpoints spread over a sphere around the
 * mesh, one square image each), reading:
 *  - view k of n looks along -u_k, u_k on the Fibonacci (golden-angle)
 *    lattice: z = 1 - (2k+1)/n, phi = k * pi (3 - sqrt 5),
 *    u = (sqrt(1 - z^2) cos phi, sqrt(1 - z^2) sin phi, z);
 *  - image axes e1 = normalize(a x u), e2 = u x e1 with a = +z, or +x when
 *    |u_z| >= 0.9;
 *  - orthographic: the res x res pixels tile the square [-R, R]^2 of the
 *    plane spanned by e1, e2 through c (c the centre of the vertex bounding
 *    box, R half its diagonal); pixel (i, j) casts the ray from
 *    c + 2R u + x e1 + y e2, x = (2 (i + 1/2) / res - 1) R,
 *    y = (2 (j + 1/2) / res - 1) R, along -u;
 *  - a face is visible when it is the first hit of at least one ray (the
 *    closest-hit rules of section 4: watertight test, no culling, ties to
 *    the lower id).
 * Exterior flood fill, reading of the normal-gated breadth-first
 * propagation: faces f and g are linked when they share an edge (two vertex
 * indices) and n_f . n_g > 0, n = (B - A) x (C - A) in double precision with
 * the operations in the order written here (the GPU evaluates the same
 * expression in the same order, so the gate is decided identically); the
 * exterior is every face linked, through any chain, to a visible face.
 */
static const double GOLDEN_ANGLE = 2.39996322972865332223;   /* pi (3 - sqrt 5) */

void or_view_basis(int k, int n, double *out) {
    double z = 1.0 - (2.0 * k + 1.0) / n;
    double r = sqrt(fmax(0.0, 1.0 - z * z));
    double phi = k * GOLDEN_ANGLE;
    d3 u = mk(r * cos(phi), r * sin(phi), z);
    d3 a = fabs(u.z) < 0.9 ? mk(0, 0, 1) : mk(1, 0, 0);
    d3 e1 = normalize(cross(a, u));
    d3 e2 = cross(u, e1);
    out[0] = u.x; out[1] = u.y; out[2] = u.z;
    out[3] = e1.x; out[4] = e1.y; out[5] = e1.z;
    out[6] = e2.x; out[7] = e2.y; out[8] = e2.z;
}

/* distance between the line o + t d (|d| = 1) and the segment a + s e,
 * s in [0, 1]; *t receives the line parameter of the closest point */
static double line_seg_dist(d3 o, d3 d, d3 a, d3 e, double *t) {
    d3 w0 = sub(a, o);
    d3 ep = sub(e, scl(d, dot(e, d)));
    d3 wp = sub(w0, scl(d, dot(w0, d)));
    double ee = dot(ep, ep);
    double s = ee > 0.0 ? -dot(wp, ep) / ee : 0.0;
    if (s < 0.0) s = 0.0;
    if (s > 1.0) s = 1.0;
    d3 q = add(a, scl(e, s));
    *t = dot(sub(q, o), d);
    return norm(sub(q, add(o, scl(d, *t))));
}

/* distance between the line and triangle tri (0 when the line meets it) */
static double line_tri_dist(const float *V, const int32_t *F, int tri, d3 o, d3 d, const ray_t *r, double *t) {
    d3 A = ldf(V, F[3 * tri]), B = ldf(V, F[3 * tri + 1]), C = ldf(V, F[3 * tri + 2]);
    double b[3];
    if (isect(r, A, B, C, t, b)) return 0.0;
    const d3 P[3] = {A, B, C};
    double best = INFINITY;
    for (int k = 0; k < 3; ++k) {
        double tk, dk = line_seg_dist(o, d, P[k], sub(P[(k + 1) % 3], P[k]), &tk);
        if (dk < best) { best = dk; *t = tk; }
    }
    return best;
}

typedef struct {
    const float *V; const int32_t *F; int64_t nf; const obvh *bvh;
    double c[3], R; int n_views, res; double delta;
    int32_t *hit; int32_t *ncand; int32_t *cand; uint8_t *edge_near;
    const int64_t *sample; int64_t nrays; int nthreads, tid;
} vis_job;

#define OR_MAX_CAND 16

static void cand_add(int32_t *list, int32_t *n, int tri) {
    for (int i = 0; i < *n && i < OR_MAX_CAND; ++i) if (list[i] == tri) return;
    if (*n < OR_MAX_CAND) list[*n] = tri;
    ++*n;
}

/* every triangle within delta of the line whose nearest approach lies no
 * later than tlim (brute force, or the BVH with boxes grown by delta) */
static void candidates(const vis_job *j, d3 o, d3 d, const ray_t *r, double tlim, int32_t *list, int32_t *n) {
    *n = 0;
    if (!j->bvh) {
        for (int64_t i = 0; i < j->nf; ++i) {
            double t, dist = line_tri_dist(j->V, j->F, (int)i, o, d, r, &t);
            if (dist <= j->delta && t <= tlim) cand_add(list, n, (int)i);
        }
        return;
    }
    const obvh *b = j->bvh;
    if (b->nf == 0) return;
    int stack[256], sp = 0;
    stack[sp++] = 0;
    while (sp) {
        const bnode *nd = &b->nodes[stack[--sp]];
        bnode g = *nd;
        for (int k = 0; k < 3; ++k) { g.lo[k] -= j->delta; g.hi[k] += j->delta; }
        double t0, t1;
        if (!box_interval(&g, o, d, &t0, &t1) || t0 > tlim) continue;
        if (nd->left < 0) {
            for (int i = nd->first; i < nd->first + nd->count; ++i) {
                int tri = b->idx[i];
                double t, dist = line_tri_dist(j->V, j->F, tri, o, d, r, &t);
                if (dist <= j->delta && t <= tlim) cand_add(list, n, tri);
            }
        } else {
            stack[sp++] = nd->left;
            stack[sp++] = nd->right;
        }
    }
}

static void vis_one(const vis_job *j, int64_t slot, int64_t ray) {
    int64_t per = (int64_t)j->res * j->res;
    int k = (int)(ray / per);
    int pix = (int)(ray % per);
    int px = pix % j->res, py = pix / j->res;
    double basis[9];
    or_view_basis(k, j->n_views, basis);
    d3 u = mk(basis[0], basis[1], basis[2]), e1 = mk(basis[3], basis[4], basis[5]), e2 = mk(basis[6], basis[7], basis[8]);
    double x = (2.0 * (px + 0.5) / j->res - 1.0) * j->R;
    double y = (2.0 * (py + 0.5) / j->res - 1.0) * j->R;
    d3 o = add(add(add(mk(j->c[0], j->c[1], j->c[2]), scl(u, 2.0 * j->R)), scl(e1, x)), scl(e2, y));
    d3 d = scl(u, -1.0);
    hit_t h;
    closest(j->V, j->F, j->nf, j->bvh, o, d, 4.0 * j->R, -1, &h);
    j->hit[slot] = h.tri;
    if (j->ncand) {
        ray_t r = make_ray(o, d);
        double tlim = (h.tri >= 0 ? h.t : 4.0 * j->R) + j->delta;
        candidates(j, o, d, &r, tlim, j->cand + slot * OR_MAX_CAND, &j->ncand[slot]);
        /* the hit point within delta of its own triangle's boundary */
        uint8_t near = 0;
        if (h.tri >= 0) {
            d3 X = add(o, scl(d, h.t));
            const int32_t *f = j->F + 3 * h.tri;
            for (int m = 0; m < 3; ++m) {
                d3 a = ldf(j->V, f[m]), e = sub(ldf(j->V, f[(m + 1) % 3]), a);
                double ee = dot(e, e), s = ee > 0 ? dot(sub(X, a), e) / ee : 0.0;
                if (s < 0) s = 0;
                if (s > 1) s = 1;
                if (norm(sub(X, add(a, scl(e, s)))) < j->delta) near = 1;
            }
        }
        j->edge_near[slot] = near;
    }
}

static void *vis_worker(void *arg) {
    vis_job *j = (vis_job *)arg;
    for (int64_t i = j->tid; i < j->nrays; i += j->nthreads) vis_one(j, i, j->sample ? j->sample[i] : i);
    return NULL;
}

/* hit [n_views*res*res]: first-hit face per ray (-1 = miss); with ncand
 * non-NULL also, per ray, the candidate faces within tol_rel*R (count in
 * ncand, up to 16 ids in cand[ray*16..]) and edge_near (hit point within
 * tol_rel*R of its triangle's boundary); visible [nf] is the union of hits.
 * With sample non-NULL only the rays sample[0..n_sample) are traced (ray id
 * = view*res*res + j*res + i), the outputs indexed by sample position, and
 * visible is the union over the sample. */
int or_visibility(const float *V, const int32_t *F, int64_t nf, void *bvh, int n_views, int res, double tol_rel,
                  int nthreads, uint8_t *visible, int32_t *hit, int32_t *ncand, int32_t *cand, uint8_t *edge_near,
                  double *frame /* out: c[3], R */, const int64_t *sample, int64_t n_sample) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t f = 0; f < nf; ++f)
        for (int m = 0; m < 3; ++m) {
            d3 p = ldf(V, F[3 * f + m]);
            for (int k = 0; k < 3; ++k) {
                double c = comp(p, k);
                if (c < lo[k]) lo[k] = c;
                if (c > hi[k]) hi[k] = c;
            }
        }
    vis_job base;
    memset(&base, 0, sizeof(base));
    base.V = V; base.F = F; base.nf = nf; base.bvh = (const obvh *)bvh;
    for (int k = 0; k < 3; ++k) base.c[k] = 0.5 * (lo[k] + hi[k]);
    base.R = 0.5 * sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                        (hi[2] - lo[2]) * (hi[2] - lo[2]));
    base.n_views = n_views; base.res = res; base.delta = tol_rel * base.R;
    base.hit = hit; base.ncand = ncand; base.cand = cand; base.edge_near = edge_near;
    base.sample = sample;
    base.nrays = sample ? n_sample : (int64_t)n_views * res * res;
    base.nthreads = nthreads;
    if (frame) { frame[0] = base.c[0]; frame[1] = base.c[1]; frame[2] = base.c[2]; frame[3] = base.R; }
    vis_job jobs[256];
    pthread_t th[256];
    for (int i = 0; i < nthreads; ++i) { jobs[i] = base; jobs[i].tid = i; }
    for (int i = 1; i < nthreads; ++i)
        if (pthread_create(&th[i], NULL, vis_worker, &jobs[i])) return -1;
    vis_worker(&jobs[0]);
    for (int i = 1; i < nthreads; ++i) pthread_join(th[i], NULL);
    memset(visible, 0, (size_t)nf);
    for (int64_t r = 0; r < base.nrays; ++r) if (hit[r] >= 0) visible[hit[r]] = 1;
    return 0;
}

/* exterior [nf] from visible [nf] by the gated flood fill above */
int or_exterior_fill(const float *V, const int32_t *F, int64_t nv, int64_t nf, const uint8_t *visible,
                     uint8_t *exterior) {
    double *nrm = (double *)malloc(sizeof(double) * 3 * (size_t)(nf > 0 ? nf : 1));
    int64_t *deg = (int64_t *)calloc((size_t)nv + 1, sizeof(int64_t));
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(nf > 0 ? nf : 1));
    int64_t *fillp = (int64_t *)calloc((size_t)nv + 1, sizeof(int64_t));
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nf > 0 ? nf : 1));
    if (!nrm || !deg || !list || !fillp || !queue) { free(nrm); free(deg); free(list); free(fillp); free(queue); return -1; }
    for (int64_t f = 0; f < nf; ++f) {
        d3 A = ldf(V, F[3 * f]), B = ldf(V, F[3 * f + 1]), C = ldf(V, F[3 * f + 2]);
        std3(nrm, f, cross(sub(B, A), sub(C, A)));
        for (int m = 0; m < 3; ++m) ++deg[F[3 * f + m] + 1];
    }
    for (int64_t v = 0; v < nv; ++v) deg[v + 1] += deg[v];
    for (int64_t f = 0; f < nf; ++f)
        for (int m = 0; m < 3; ++m) { int32_t v = F[3 * f + m]; list[deg[v] + fillp[v]++] = (int32_t)f; }
    int64_t qh = 0, qt = 0;
    for (int64_t f = 0; f < nf; ++f) {
        exterior[f] = visible[f] ? 1 : 0;
        if (exterior[f]) queue[qt++] = (int32_t)f;
    }
    while (qh < qt) {
        int32_t f = queue[qh++];
        d3 nf_ = ldd(nrm, f);
        for (int m = 0; m < 3; ++m) {
            int32_t a = F[3 * f + m], b = F[3 * f + (m + 1) % 3];
            if (a == b) continue;
            for (int64_t i = deg[a]; i < deg[a + 1]; ++i) {
                int32_t g = list[i];
                if (g == f || exterior[g]) continue;
                if (F[3 * g] != b && F[3 * g + 1] != b && F[3 * g + 2] != b) continue;
                if (dot(nf_, ldd(nrm, g)) > 0.0) { exterior[g] = 1; queue[qt++] = g; }
            }
        }
    }
    free(nrm); free(deg); free(list); free(fillp); free(queue);
    return 0;
}

/* ------------------------------------------------- 9. QEM simplification (Sec. 6.1)
 * Quadric-error edge collapse with the paper's placement rule, in rounds of
 * independent collapses.  Everything is double precision with the
 * operations in the order written (the GPU evaluates the same expressions
 * in the same order, so every decision below is taken identically).
 *
 * Quadrics.  Face f with corners P0, P1, P2: n = (P1 - P0) x (P2 - P0),
 * unit normal m = n / |n| (no plane for |n| = 0), d = -(m . P0),
 * p = (m, d), K_f = p p^T.  Q_v = sum of K_f over the faces incident to v,
 * in increasing face id.  Merging an edge (a, b) gives Q = Q_a + Q_b, and
 * after the collapse the kept vertex carries that Q.  E(v) = [v 1] Q [v 1]^T.
 *
 * Placement (paper): for an interior edge, x = -A^-1 b with A the upper-left
 * 3x3 of Q and b its upper-right column; t = <x - v0, v1 - v0> / |v1 - v0|^2
 * clamped to [0, 1]; v = v0 + t (v1 - v0).  Readings: A is singular when
 * |det A| <= 1e-12 * max_i |A_ii|^3, and then t = 1/2 (the midpoint); the
 * inverse is the adjugate over the determinant.  Boundary edges (one
 * incident face) go to the endpoint with the lower E (ties to v0); an
 * interior edge with one boundary endpoint goes to that endpoint; an
 * interior edge with two boundary endpoints is not collapsed.  The cost is
 * E(v), negative rounding clamped to 0.  With `midpoint` set, interior edges
 * go to their midpoint instead (the baseline the paper improves on).
 *
 * Validity (readings): the edge has at most two faces; both endpoints have
 * at most 64 neighbours; the link condition
 * |N(a) ∩ N(b)| = number of faces on the edge; the union of the two
 * neighbourhoods has more than 4 vertices (no tetrahedron collapses); and
 * no surviving face around a or b turns over: n_old . n_new > 0.
 *
 * Rounds (our reading of collapsing many edges at once): the unique edges (a < b) are
 * ranked in (a, b) order; key = (bits of the cost rounded to float32) << 32
 * | rank.  m1(v) = min key of the valid edges at v, m2(v) = min of m1 over v
 * and its neighbours; edge (a, b) collapses when key = m2(a) = m2(b).  Two
 * such edges never touch adjacent vertices, so their collapses are
 * independent.  A round that would go below the target keeps only its
 * smallest keys, just enough to reach it.  Collapsing (a, b) keeps a at v,
 * removes b, drops the faces holding both and renames b to a in the others.
 * It stops at the target face count or when no edge collapses. */
typedef struct { double q[10]; } qem_quad;   /* q00 q01 q02 q03 q11 q12 q13 q22 q23 q33 */

static void face_quadric(d3 P0, d3 P1, d3 P2, qem_quad *K, int *ok) {
    d3 n = cross(sub(P1, P0), sub(P2, P0));
    double len = sqrt(dot(n, n));
    memset(K, 0, sizeof(*K));
    *ok = len > 0.0;
    if (!*ok) return;
    d3 m = mk(n.x / len, n.y / len, n.z / len);
    double p[4] = {m.x, m.y, m.z, -dot(m, P0)};
    int k = 0;
    for (int i = 0; i < 4; ++i)
        for (int j = i; j < 4; ++j) K->q[k++] = p[i] * p[j];
}

static double quad_eval(const qem_quad *Q, d3 v) {
    const double *q = Q->q;
    double e = q[0] * v.x * v.x;
    e = e + 2.0 * q[1] * v.x * v.y;
    e = e + 2.0 * q[2] * v.x * v.z;
    e = e + 2.0 * q[3] * v.x;
    e = e + q[4] * v.y * v.y;
    e = e + 2.0 * q[5] * v.y * v.z;
    e = e + 2.0 * q[6] * v.y;
    e = e + q[7] * v.z * v.z;
    e = e + 2.0 * q[8] * v.z;
    e = e + q[9];
    return e;
}

/* placement of the interior edge v0 -> v1 under Q; returns t */
static double qem_place(const qem_quad *Q, d3 v0, d3 v1, int *singular) {
    const double *q = Q->q;
    double a00 = q[0], a01 = q[1], a02 = q[2], a11 = q[4], a12 = q[5], a22 = q[7];
    double b0 = q[3], b1 = q[6], b2 = q[8];
    double c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
    double c11 = a00 * a22 - a02 * a02, c12 = a01 * a02 - a00 * a12, c22 = a00 * a11 - a01 * a01;
    double det = a00 * c00 + a01 * c01 + a02 * c02;
    double s = fmax(fabs(a00), fmax(fabs(a11), fabs(a22)));
    *singular = !(fabs(det) > 1e-12 * s * s * s);
    if (*singular) return 0.5;
    d3 x = mk(-(c00 * b0 + c01 * b1 + c02 * b2) / det, -(c01 * b0 + c11 * b1 + c12 * b2) / det,
              -(c02 * b0 + c12 * b1 + c22 * b2) / det);
    d3 e = sub(v1, v0);
    double ee = dot(e, e);
    if (!(ee > 0.0)) return 0.0;
    double t = dot(sub(x, v0), e) / ee;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    return t;
}

static uint64_t qem_key(double cost, uint32_t rank) {
    float c = (float)(cost > 0.0 ? cost : 0.0);
    uint32_t bits;
    memcpy(&bits, &c, 4);
    return ((uint64_t)bits << 32) | rank;
}

typedef struct { int32_t a, b; int nfaces; } qedge_t;

#define QEM_MAX_NBR 64

static int qedge_cmp(const void *x, const void *y) {
    const qedge_t *p = (const qedge_t *)x, *q = (const qedge_t *)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    return 0;
}

static int u64_cmp(const void *x, const void *y) {
    uint64_t p = *(const uint64_t *)x, q = *(const uint64_t *)y;
    return p < q ? -1 : (p > q ? 1 : 0);
}

static int face_has(const int32_t *F, int64_t f, int32_t v) { return F[3 * f] == v || F[3 * f + 1] == v || F[3 * f + 2] == v; }

/* V [nv*3] double, F [nf*3] int32 are updated in place; alive flags out;
 * returns the number of rounds, -1 on allocation failure.  stats (optional,
 * [max_rounds*2]): alive faces and collapses per round. */
int or_qem_simplify(double *V, int64_t nv, int32_t *F, int64_t nf, int64_t target, uint8_t *valive, uint8_t *falive,
                    int max_rounds, int64_t *stats, int midpoint) {
    qem_quad *Q = (qem_quad *)calloc((size_t)nv, sizeof(qem_quad));
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nv + 1));
    int32_t *vf = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)nf);
    int64_t *fillc = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
    qedge_t *E = (qedge_t *)malloc(sizeof(qedge_t) * 3 * (size_t)nf);
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * 3 * (size_t)nf);
    double *tpos = (double *)malloc(sizeof(double) * 3 * 3 * (size_t)nf);
    uint64_t *m1 = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)nv);
    uint64_t *m2 = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)nv);
    uint8_t *bnd = (uint8_t *)malloc((size_t)nv);
    int32_t *remap = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    int32_t *nbr_a = (int32_t *)malloc(sizeof(int32_t) * (QEM_MAX_NBR + 1)),
            *nbr_b = (int32_t *)malloc(sizeof(int32_t) * (QEM_MAX_NBR + 1));
    uint64_t *selk = (uint64_t *)malloc(sizeof(uint64_t) * 3 * (size_t)nf);
    if (!Q || !off || !vf || !fillc || !E || !key || !tpos || !m1 || !m2 || !bnd || !remap || !nbr_a || !nbr_b || !selk) {
        free(Q); free(off); free(vf); free(fillc); free(E); free(key); free(tpos); free(m1); free(m2); free(bnd);
        free(remap); free(nbr_a); free(nbr_b); free(selk);
        return -1;
    }
    /* faces with a repeated vertex index are dropped; vertices of no face are not alive */
    int64_t alive = 0;
    for (int64_t v = 0; v < nv; ++v) valive[v] = 0;
    for (int64_t f = 0; f < nf; ++f) {
        falive[f] = !(F[3 * f] == F[3 * f + 1] || F[3 * f + 1] == F[3 * f + 2] || F[3 * f] == F[3 * f + 2]);
        if (!falive[f]) continue;
        ++alive;
        for (int k = 0; k < 3; ++k) valive[F[3 * f + k]] = 1;
    }
    /* initial quadrics: faces in increasing id at every vertex */
    for (int64_t f = 0; f < nf; ++f) {
        if (!falive[f]) continue;
        qem_quad K;
        int ok;
        face_quadric(ldd(V, F[3 * f]), ldd(V, F[3 * f + 1]), ldd(V, F[3 * f + 2]), &K, &ok);
        if (!ok) continue;
        for (int k = 0; k < 3; ++k) {
            qem_quad *q = &Q[F[3 * f + k]];
            for (int i = 0; i < 10; ++i) q->q[i] = q->q[i] + K.q[i];
        }
    }
    int round = 0;
    while (alive > target && round < max_rounds) {
        /* vertex -> alive faces, increasing face id */
        for (int64_t v = 0; v <= nv; ++v) off[v] = 0;
        for (int64_t f = 0; f < nf; ++f)
            if (falive[f]) for (int k = 0; k < 3; ++k) ++off[F[3 * f + k] + 1];
        for (int64_t v = 0; v < nv; ++v) { off[v + 1] += off[v]; fillc[v] = 0; }
        for (int64_t f = 0; f < nf; ++f)
            if (falive[f]) for (int k = 0; k < 3; ++k) { int32_t v = F[3 * f + k]; vf[off[v] + fillc[v]++] = (int32_t)f; }
        /* unique edges in (a, b) order with their face counts */
        int64_t ne = 0;
        for (int64_t f = 0; f < nf; ++f) {
            if (!falive[f]) continue;
            for (int k = 0; k < 3; ++k) {
                int32_t a = F[3 * f + k], b = F[3 * f + (k + 1) % 3];
                qedge_t e = {a < b ? a : b, a < b ? b : a, 1};
                E[ne++] = e;
            }
        }
        qsort(E, (size_t)ne, sizeof(qedge_t), qedge_cmp);
        int64_t nu = 0;
        for (int64_t i = 0; i < ne; ++i) {
            if (nu > 0 && E[nu - 1].a == E[i].a && E[nu - 1].b == E[i].b) { E[nu - 1].nfaces++; continue; }
            E[nu++] = E[i];
        }
        for (int64_t v = 0; v < nv; ++v) bnd[v] = 0;
        for (int64_t i = 0; i < nu; ++i) if (E[i].nfaces == 1) { bnd[E[i].a] = 1; bnd[E[i].b] = 1; }
        /* cost, placement and validity of every edge */
        for (int64_t i = 0; i < nu; ++i) {
            int32_t a = E[i].a, b = E[i].b;
            key[i] = UINT64_MAX;
            if (E[i].nfaces > 2) continue;
            qem_quad Qe;
            for (int k = 0; k < 10; ++k) Qe.q[k] = Q[a].q[k] + Q[b].q[k];
            d3 va = ldd(V, a), vb = ldd(V, b), v;
            if (E[i].nfaces == 1) {
                v = quad_eval(&Qe, vb) < quad_eval(&Qe, va) ? vb : va;
            } else if (bnd[a] && bnd[b]) {
                continue;
            } else if (bnd[a]) {
                v = va;
            } else if (bnd[b]) {
                v = vb;
            } else {
                int sing;
                double t = midpoint ? 0.5 : qem_place(&Qe, va, vb, &sing);
                v = add(va, scl(sub(vb, va), t));
            }
            /* neighbourhoods */
            int na = 0, nb = 0;
            for (int64_t j = off[a]; j < off[a + 1]; ++j)
                for (int k = 0; k < 3; ++k) {
                    int32_t u = F[3 * vf[j] + k];
                    if (u == a) continue;
                    int seen = 0;
                    for (int m = 0; m < na; ++m) if (nbr_a[m] == u) seen = 1;
                    if (!seen && na <= QEM_MAX_NBR) nbr_a[na++] = u;
                }
            for (int64_t j = off[b]; j < off[b + 1]; ++j)
                for (int k = 0; k < 3; ++k) {
                    int32_t u = F[3 * vf[j] + k];
                    if (u == b) continue;
                    int seen = 0;
                    for (int m = 0; m < nb; ++m) if (nbr_b[m] == u) seen = 1;
                    if (!seen && nb <= QEM_MAX_NBR) nbr_b[nb++] = u;
                }
            if (na > QEM_MAX_NBR || nb > QEM_MAX_NBR) continue;
            int common = 0;
            for (int m = 0; m < na; ++m)
                for (int n = 0; n < nb; ++n) if (nbr_a[m] == nbr_b[n]) ++common;
            if (common != E[i].nfaces) continue;
            if (na + nb - common <= 4) continue;   /* |N(a) ∪ N(b)| counting a and b: na + nb - common */
            /* no surviving face turns over */
            int flip = 0;
            for (int side = 0; side < 2 && !flip; ++side) {
                int32_t w = side ? b : a, o = side ? a : b;
                for (int64_t j = off[w]; j < off[w + 1] && !flip; ++j) {
                    int64_t g = vf[j];
                    if (face_has(F, g, o)) continue;
                    d3 P[3], R[3];
                    for (int k = 0; k < 3; ++k) {
                        P[k] = ldd(V, F[3 * g + k]);
                        R[k] = F[3 * g + k] == w ? v : P[k];
                    }
                    d3 n0 = cross(sub(P[1], P[0]), sub(P[2], P[0]));
                    d3 n1 = cross(sub(R[1], R[0]), sub(R[2], R[0]));
                    if (!(dot(n0, n1) > 0.0)) flip = 1;
                }
            }
            if (flip) continue;
            key[i] = qem_key(quad_eval(&Qe, v), (uint32_t)i);
            std3(tpos, i, v);
        }
        /* two-ring minima */
        for (int64_t v = 0; v < nv; ++v) m1[v] = UINT64_MAX;
        for (int64_t i = 0; i < nu; ++i) {
            if (key[i] < m1[E[i].a]) m1[E[i].a] = key[i];
            if (key[i] < m1[E[i].b]) m1[E[i].b] = key[i];
        }
        for (int64_t v = 0; v < nv; ++v) m2[v] = m1[v];
        for (int64_t i = 0; i < nu; ++i) {
            if (m1[E[i].b] < m2[E[i].a]) m2[E[i].a] = m1[E[i].b];
            if (m1[E[i].a] < m2[E[i].b]) m2[E[i].b] = m1[E[i].a];
        }
        int64_t nsel = 0, removable = 0;
        for (int64_t i = 0; i < nu; ++i)
            if (key[i] != UINT64_MAX && key[i] == m2[E[i].a] && key[i] == m2[E[i].b]) {
                selk[nsel++] = key[i];
                removable += E[i].nfaces;
            }
        if (nsel == 0) break;
        uint64_t limit = UINT64_MAX;
        if (alive - removable < target) {
            qsort(selk, (size_t)nsel, sizeof(uint64_t), u64_cmp);
            int64_t gone = 0;
            for (int64_t s = 0; s < nsel; ++s) {
                gone += E[(uint32_t)selk[s]].nfaces;
                if (alive - gone <= target) { limit = selk[s]; break; }
            }
        }
        /* collapse */
        for (int64_t v = 0; v < nv; ++v) remap[v] = (int32_t)v;
        int64_t ncol = 0;
        for (int64_t i = 0; i < nu; ++i) {
            if (key[i] == UINT64_MAX || key[i] != m2[E[i].a] || key[i] != m2[E[i].b] || key[i] > limit) continue;
            int32_t a = E[i].a, b = E[i].b;
            std3(V, a, ldd(tpos, i));
            for (int k = 0; k < 10; ++k) Q[a].q[k] = Q[a].q[k] + Q[b].q[k];
            valive[b] = 0;
            remap[b] = a;
            ++ncol;
        }
        for (int64_t f = 0; f < nf; ++f) {
            if (!falive[f]) continue;
            int32_t r[3];
            for (int k = 0; k < 3; ++k) r[k] = remap[F[3 * f + k]];
            if (r[0] == r[1] || r[1] == r[2] || r[0] == r[2]) { falive[f] = 0; --alive; continue; }
            for (int k = 0; k < 3; ++k) F[3 * f + k] = r[k];
        }
        if (stats) { stats[2 * round] = alive; stats[2 * round + 1] = ncol; }
        ++round;
    }
    free(Q); free(off); free(vf); free(fillc); free(E); free(key); free(tpos); free(m1); free(m2); free(bnd);
    free(remap); free(nbr_a); free(nbr_b); free(selk);
    return round;
}

/* pieces exposed for pin tests */
void or_qem_face_quadric(const double *P, double *q) {
    qem_quad K;
    int ok;
    face_quadric(ldd(P, 0), ldd(P, 1), ldd(P, 2), &K, &ok);
    memcpy(q, K.q, sizeof(K.q));
}

double or_qem_eval(const double *q, const double *v) {
    qem_quad Q;
    memcpy(Q.q, q, sizeof(Q.q));
    return quad_eval(&Q, mk(v[0], v[1], v[2]));
}

double or_qem_place(const double *q, const double *v0, const double *v1, int *singular) {
    qem_quad Q;
    memcpy(Q.q, q, sizeof(Q.q));
    return qem_place(&Q, mk(v0[0], v0[1], v0[2]), mk(v1[0], v1[1], v1[2]), singular);
}

/* ------------------------------------------------- 10. UV-space backprojection (Sec. 7.4)
 * Readings.  A view is a pinhole camera with world -> camera rotation R (rows
 * right, down, forward), translation t and intrinsics fx, fy, cx, cy in
 * pixels: a point p has camera coordinates c = R p + t, depth z = c.z, and
 * image position u = fx c.x / z + cx, v = fy c.y / z + cy; pixel (i, j)
 * covers [i, i+1) x [j, j+1).
 *  - Depth buffer: for every pixel, the first hit of the ray through its
 *    centre in front of the camera (the smallest t > 0 under section 4's
 *    intersection test, equal t: the lower triangle id), its depth z and
 *    world point; +inf / NaN where the ray misses.  A pixel is an edge pixel
 *    when it is a hit and one of its 4-neighbours is a miss or has a world
 *    point farther than edge_tol from its own (the paper's large
 *    neighbour differences of the point map).
 *  - Per ray texel (the raster of section 2, surface point p = sum b_i v_i,
 *    normal n = normalize(sum b_i n_i) of the smooth vertex normals): for
 *    every view with z > 0 and (u, v) inside the image, the pixel (floor u,
 *    floor v) must be a hit, not an edge pixel, with z <= its depth +
 *    depth_tol; then I = max(0, n . normalize(C - p)) (C the camera centre)
 *    and the colour A is the bilinear sample of the view's RGB at
 *    (u - 1/2, v - 1/2), clamped to the image, 8-bit codes / 255.
 *  - Blend: T = sum_k w_k I_k^alpha A_k / (sum_k w_k I_k^alpha + eps) over the
 *    views with I_k > 0, evaluated through the log-sum-exp form
 *    m = max_k (log w_k + alpha log I_k),
 *    T = sum_k e^(L_k - m) A_k / (sum_k e^(L_k - m) + eps e^(-m)).
 *    A texel with no such view stays unfilled (T = 0).
 *  - Exception flags: a texel is flagged when, for some view, u or v lies
 *    within 1e-3 pixel of a pixel boundary or of the image border, z lies
 *    within 1e-5 * scale of the depth limit, a neighbour distance of the
 *    pixel lies within 1e-5 * scale of edge_tol, or the pixel or one of its
 *    4-neighbours is a rounding-dependent render (or_render_view's near). */
typedef struct { double R[9], t[3], fx, fy, cx, cy; } cam_t;

static cam_t load_cam(const float *c) {
    cam_t k;
    for (int i = 0; i < 9; ++i) k.R[i] = c[i];
    for (int i = 0; i < 3; ++i) k.t[i] = c[9 + i];
    k.fx = c[12]; k.fy = c[13]; k.cx = c[14]; k.cy = c[15];
    return k;
}

static d3 cam_apply(const cam_t *k, d3 p) {
    return mk(k->R[0] * p.x + k->R[1] * p.y + k->R[2] * p.z + k->t[0],
              k->R[3] * p.x + k->R[4] * p.y + k->R[5] * p.z + k->t[1],
              k->R[6] * p.x + k->R[7] * p.y + k->R[8] * p.z + k->t[2]);
}

static d3 cam_centre(const cam_t *k) {   /* C = -R^T t */
    return mk(-(k->R[0] * k->t[0] + k->R[3] * k->t[1] + k->R[6] * k->t[2]),
              -(k->R[1] * k->t[0] + k->R[4] * k->t[1] + k->R[7] * k->t[2]),
              -(k->R[2] * k->t[0] + k->R[5] * k->t[1] + k->R[8] * k->t[2]));
}

/* the first hit in front of the origin: the smallest t > 0 over the
 * triangles the line meets (equal t: the lower triangle id) */
static void first_hit(const float *V, const int32_t *F, const obvh *b, d3 o, d3 d, hit_t *best) {
    ray_t r = make_ray(o, d);
    best->tri = -1; best->t = INFINITY; best->b[0] = best->b[1] = best->b[2] = 0.0;
    if (b->nf == 0) return;
    int stack[256], sp = 0;
    stack[sp++] = 0;
    while (sp) {
        const bnode *n = &b->nodes[stack[--sp]];
        double t0, t1;
        if (!box_interval(n, o, d, &t0, &t1)) continue;
        if (t1 < 0.0 || t0 > best->t) continue;
        if (n->left < 0) {
            for (int i = n->first; i < n->first + n->count; ++i) {
                int tri = b->idx[i];
                double t, bb[3];
                if (!isect(&r, ldf(V, F[3 * tri]), ldf(V, F[3 * tri + 1]), ldf(V, F[3 * tri + 2]), &t, bb)) continue;
                if (!(t > 0.0)) continue;
                if (t < best->t || (t == best->t && tri < best->tri)) {
                    best->tri = tri; best->t = t; best->b[0] = bb[0]; best->b[1] = bb[1]; best->b[2] = bb[2];
                }
            }
        } else {
            stack[sp++] = n->left;
            stack[sp++] = n->right;
        }
    }
}

/* depth [h*w] (camera z of the first hit, +inf on a miss), point [h*w*3]
 * (NaN on a miss), near [h*w] per view: the pixel's value depends on
 * rounding: its ray misses but passes within tol of a triangle, or passes
 * within tol of a triangle 100 tol or more in front of its hit, or (where
 * the ray can leave the hit's sheet within tol of the hit) behind it */
int or_render_view(const float *V, const int32_t *F, int64_t nf, void *bvh, const float *camf, int w, int h,
                   double tol, double *depth, double *point, uint8_t *near) {
    cam_t k = load_cam(camf);
    d3 C = cam_centre(&k);
    const obvh *b = (const obvh *)bvh;
    for (int j = 0; j < h; ++j)
        for (int i = 0; i < w; ++i) {
            int64_t px = (int64_t)j * w + i;
            d3 dc = mk((i + 0.5 - k.cx) / k.fx, (j + 0.5 - k.cy) / k.fy, 1.0);
            /* world direction R^T dc */
            d3 d = normalize(mk(k.R[0] * dc.x + k.R[3] * dc.y + k.R[6] * dc.z,
                                k.R[1] * dc.x + k.R[4] * dc.y + k.R[7] * dc.z,
                                k.R[2] * dc.x + k.R[5] * dc.y + k.R[8] * dc.z));
            hit_t hh;
            first_hit(V, F, b, C, d, &hh);
            /* triangles within tol of the ray (those behind the camera plane
             * by more than 100 tol play no part) */
            vis_job vj;
            memset(&vj, 0, sizeof(vj));
            vj.V = V; vj.F = F; vj.nf = nf; vj.bvh = b; vj.delta = tol;
            int32_t cl[OR_MAX_CAND], nc = 0;
            ray_t r = make_ray(C, d);
            int hit = hh.tri >= 0;
            candidates(&vj, C, d, &r, 1e30, cl, &nc);
            const double sep = 100.0 * tol;
            {
                int kept = 0;
                for (int m = 0; m < nc && m < OR_MAX_CAND; ++m) {
                    double tc;
                    line_tri_dist(V, F, cl[m], C, d, &r, &tc);
                    if (tc >= -sep) cl[kept++] = cl[m];
                }
                if (nc <= OR_MAX_CAND) nc = kept;
            }
            uint8_t nr = 0;
            if (hit) {
                d3 X = add(C, scl(d, hh.t));
                depth[px] = cam_apply(&k, X).z;
                std3(point, px, X);
                /* a silhouette: a triangle within tol of the ray clearly in front
                 * of the hit, or clearly behind it while the ray can leave the
                 * hit's sheet within tol of the hit: the hit lies within tol of
                 * an edge of its triangle that no same-facing triangle continues,
                 * or a triangle near the hit faces the other way.  Across an edge
                 * that a same-facing triangle continues, rounding only moves the
                 * hit to that neighbour: depth and point stay. */
                const int32_t *f = F + 3 * hh.tri;
                d3 nh = cross(sub(ldf(V, f[1]), ldf(V, f[0])), sub(ldf(V, f[2]), ldf(V, f[0])));
                double sh = dot(d, nh);
                int leave = 0;
                for (int m = 0; m < 3 && !leave; ++m) {
                    d3 a = ldf(V, f[m]), e = sub(ldf(V, f[(m + 1) % 3]), a);
                    double ee = dot(e, e), sp = ee > 0 ? dot(sub(X, a), e) / ee : 0.0;
                    if (sp < 0) sp = 0;
                    if (sp > 1) sp = 1;
                    if (!(norm(sub(X, add(a, scl(e, sp)))) < tol)) continue;
                    int cont = 0;
                    for (int q = 0; q < nc && q < OR_MAX_CAND; ++q) {
                        const int32_t *g = F + 3 * cl[q];
                        if (cl[q] == hh.tri) continue;
                        int ha = 0, hb = 0;
                        for (int z = 0; z < 3; ++z) {
                            ha |= g[z] == f[m];
                            hb |= g[z] == f[(m + 1) % 3];
                        }
                        if (!(ha && hb)) continue;
                        d3 ng = cross(sub(ldf(V, g[1]), ldf(V, g[0])), sub(ldf(V, g[2]), ldf(V, g[0])));
                        if (dot(d, ng) * sh > 0) cont = 1;
                    }
                    if (!cont) leave = 1;
                }
                for (int m = 0; m < nc && m < OR_MAX_CAND; ++m) {
                    double tc;
                    line_tri_dist(V, F, cl[m], C, d, &r, &tc);
                    if (tc < hh.t - sep) nr = 1;
                    if (fabs(tc - hh.t) <= sep) {
                        const int32_t *g = F + 3 * cl[m];
                        d3 ng = cross(sub(ldf(V, g[1]), ldf(V, g[0])), sub(ldf(V, g[2]), ldf(V, g[0])));
                        if (!(dot(d, ng) * sh > 0)) leave = 1;
                    }
                }
                if (leave)
                    for (int m = 0; m < nc && m < OR_MAX_CAND; ++m) {
                        double tc;
                        line_tri_dist(V, F, cl[m], C, d, &r, &tc);
                        if (tc > hh.t + sep) nr = 1;
                    }
                if (nc > OR_MAX_CAND) nr = 1;
            } else {
                depth[px] = INFINITY;
                std3(point, px, mk(NAN, NAN, NAN));
                if (nc > 0) nr = 1;   /* a miss near the silhouette */
            }
            near[px] = nr;
        }
    return 0;
}

static double bilinear(const uint8_t *img, int w, int h, int ch, double x, double y) {
    double fx = floor(x), fy = floor(y);
    double ax = x - fx, ay = y - fy;
    int x0 = (int)fx, y0 = (int)fy;
    double acc = 0.0;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
            int xx = x0 + dx, yy = y0 + dy;
            if (xx < 0) xx = 0;
            if (yy < 0) yy = 0;
            if (xx > w - 1) xx = w - 1;
            if (yy > h - 1) yy = h - 1;
            double wgt = (dx ? ax : 1.0 - ax) * (dy ? ay : 1.0 - ay);
            acc += wgt * (img[((int64_t)yy * w + xx) * 4 + ch] / 255.0);
        }
    return acc;
}

/* --- anisotropic filtering (Sec. 7.4), readings:
 *  - Mip chain of each view's RGB (codes / 255): level l+1 has max(1, w_l / 2) x max(1, h_l / 2)
 *    pixels; its pixel j is centred at level-l coordinate 2j + 1, and takes the 8 level-l pixels
 *    i = 2j - 3 .. 2j + 4 (clamped to the image) with weights L((i + 1/2 - (2j + 1)) / 2),
 *    L(x) = sinc(x) sinc(x / 2) for |x| < 2 (Lanczos-2 stretched for a 2x reduction),
 *    normalised; rows first, then columns; the level is clamped to [0, 1].
 *  - Per-level sharpening: level l >= 1 is sampled as clamp(P + s (P - B P), 0, 1), B the
 *    separable [1, 2, 1] / 4 blur with clamped borders; P is the unsharpened level, from which
 *    the next level is built.
 *  - Footprint: the texel's surface point moves by dp/dx, dp/dy per texel (the owning face's
 *    affine UV -> position map); the Jacobian J of texel -> image is the central difference of
 *    the projections of p -+ dp/dx / 2 and p -+ dp/dy / 2.  A face whose UV area is below
 *    1e-4 texel^2, or a difference point behind the camera, falls back to the centre sample.
 *  - SVD of J: singular values s1 >= s2 and the major image direction e1 (from J J^T).
 *    Taps N = clamp(ceil(s1 / s2 - 0.05), 1, max_taps) (ratios within 5 % above an integer add
 *    no tap, so an isotropic footprint keeps one tap under rounding), spread over the major axis:
 *    (u, v) + e1 s1 ((i + 1/2) / N - 1/2), equally weighted.
 *  - Level lambda = log2(max(s2, s1 / max_taps)) + lod_bias (the minor axis, raised when the taps
 *    cannot cover the major axis), clamped to [0, levels - 1]; trilinear: the bilinear samples of
 *    levels floor(lambda) and floor(lambda) + 1 at (u / 2^l - 1/2, v / 2^l - 1/2), blended by the
 *    fraction; level 0 is the 8-bit image itself. */
#define OR_MAX_LEV 16
typedef struct { int n; int w[OR_MAX_LEV], h[OR_MAX_LEV]; double *p[OR_MAX_LEV], *s[OR_MAX_LEV]; } mips_t;

static double lanczos2(double x) {
    if (x == 0.0) return 1.0;
    if (fabs(x) >= 2.0) return 0.0;
    const double px = M_PI * x;
    return 2.0 * sin(px) * sin(0.5 * px) / (px * px);
}

/* level 0 of pyramid m is the image (never stored); levels 1.. are built here */
static int build_mips(const uint8_t *img, int w, int h, double sharpen, mips_t *m) {
    memset(m, 0, sizeof(*m));
    m->n = 1;
    m->w[0] = w; m->h[0] = h;
    double wt[8], sw = 0.0;
    for (int t = 0; t < 8; ++t) { wt[t] = lanczos2((t - 3.5) / 2.0); sw += wt[t]; }
    for (int t = 0; t < 8; ++t) wt[t] /= sw;
    const double *prev = NULL;
    int pw = w, ph = h;
    while ((pw > 1 || ph > 1) && m->n < OR_MAX_LEV) {
        int nw = pw / 2 > 1 ? pw / 2 : 1, nh = ph / 2 > 1 ? ph / 2 : 1;
        double *tmp = (double *)malloc(sizeof(double) * 3 * (size_t)nw * ph);
        double *out = (double *)malloc(sizeof(double) * 3 * (size_t)nw * nh);
        double *shp = (double *)malloc(sizeof(double) * 3 * (size_t)nw * nh);
        double *blr = (double *)malloc(sizeof(double) * 3 * (size_t)nw * nh);
        if (!tmp || !out || !shp || !blr) { free(tmp); free(out); free(shp); free(blr); return -1; }
        for (int y = 0; y < ph; ++y)
            for (int x = 0; x < nw; ++x)
                for (int c = 0; c < 3; ++c) {
                    double acc = 0.0;
                    for (int t = 0; t < 8; ++t) {
                        int i = 2 * x - 3 + t;
                        if (i < 0) i = 0;
                        if (i > pw - 1) i = pw - 1;
                        double v = prev ? prev[((size_t)y * pw + i) * 3 + c] : img[((size_t)y * pw + i) * 4 + c] / 255.0;
                        acc += wt[t] * v;
                    }
                    tmp[((size_t)y * nw + x) * 3 + c] = acc;
                }
        for (int y = 0; y < nh; ++y)
            for (int x = 0; x < nw; ++x)
                for (int c = 0; c < 3; ++c) {
                    double acc = 0.0;
                    for (int t = 0; t < 8; ++t) {
                        int j = 2 * y - 3 + t;
                        if (j < 0) j = 0;
                        if (j > ph - 1) j = ph - 1;
                        acc += wt[t] * tmp[((size_t)j * nw + x) * 3 + c];
                    }
                    out[((size_t)y * nw + x) * 3 + c] = acc < 0.0 ? 0.0 : (acc > 1.0 ? 1.0 : acc);
                }
        /* sharpened copy: P + s (P - B P) */
        for (int y = 0; y < nh; ++y)
            for (int x = 0; x < nw; ++x)
                for (int c = 0; c < 3; ++c) {
                    int xl = x > 0 ? x - 1 : 0, xr = x < nw - 1 ? x + 1 : nw - 1;
                    blr[((size_t)y * nw + x) * 3 + c] = 0.25 * out[((size_t)y * nw + xl) * 3 + c] +
                                                        0.5 * out[((size_t)y * nw + x) * 3 + c] +
                                                        0.25 * out[((size_t)y * nw + xr) * 3 + c];
                }
        for (int y = 0; y < nh; ++y)
            for (int x = 0; x < nw; ++x)
                for (int c = 0; c < 3; ++c) {
                    int yu = y > 0 ? y - 1 : 0, yd = y < nh - 1 ? y + 1 : nh - 1;
                    double b = 0.25 * blr[((size_t)yu * nw + x) * 3 + c] + 0.5 * blr[((size_t)y * nw + x) * 3 + c] +
                               0.25 * blr[((size_t)yd * nw + x) * 3 + c];
                    double P = out[((size_t)y * nw + x) * 3 + c];
                    double v = P + sharpen * (P - b);
                    shp[((size_t)y * nw + x) * 3 + c] = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
                }
        free(tmp);
        free(blr);
        m->p[m->n] = out; m->s[m->n] = shp; m->w[m->n] = nw; m->h[m->n] = nh;
        ++m->n;
        prev = out; pw = nw; ph = nh;
    }
    return 0;
}

static void free_mips(mips_t *m) {
    for (int l = 1; l < m->n; ++l) { free(m->p[l]); free(m->s[l]); }
}

static double bilinear_d(const double *lev, int w, int h, int ch, double x, double y) {
    double fx = floor(x), fy = floor(y);
    double ax = x - fx, ay = y - fy;
    int x0 = (int)fx, y0 = (int)fy;
    double acc = 0.0;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
            int xx = x0 + dx, yy = y0 + dy;
            if (xx < 0) xx = 0;
            if (yy < 0) yy = 0;
            if (xx > w - 1) xx = w - 1;
            if (yy > h - 1) yy = h - 1;
            acc += (dx ? ax : 1.0 - ax) * (dy ? ay : 1.0 - ay) * lev[((int64_t)yy * w + xx) * 3 + ch];
        }
    return acc;
}

/* the bilinear sample of level l at level-0 image position (u, v) */
static double level_sample(const uint8_t *img, const mips_t *m, int l, int ch, double u, double v) {
    if (l == 0) return bilinear(img, m->w[0], m->h[0], ch, u - 0.5, v - 0.5);
    const double sc = ldexp(1.0, -l);
    return bilinear_d(m->s[l], m->w[l], m->h[l], ch, u * sc - 0.5, v * sc - 0.5);
}

static double trilinear(const uint8_t *img, const mips_t *m, double lam, int ch, double u, double v) {
    int l0 = (int)floor(lam);
    double f = lam - l0;
    if (l0 >= m->n - 1) return level_sample(img, m, m->n - 1, ch, u, v);
    double a = level_sample(img, m, l0, ch, u, v);
    if (f == 0.0) return a;
    return (1.0 - f) * a + f * level_sample(img, m, l0 + 1, ch, u, v);
}

/* edge pixel test; *amb is set when a neighbour distance lies within
 * amb_tol of edge_tol (the decision is a rounding decision there) */
static int is_edge(const double *depth, const double *point, int w, int h, int i, int j, double edge_tol,
                   double amb_tol, int *amb) {
    int64_t px = (int64_t)j * w + i;
    if (!(depth[px] < INFINITY)) return 0;
    const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
    int e = 0;
    for (int n = 0; n < 4; ++n) {
        int ii = i + di[n], jj = j + dj[n];
        if (ii < 0 || jj < 0 || ii >= w || jj >= h) continue;
        int64_t q = (int64_t)jj * w + ii;
        if (!(depth[q] < INFINITY)) { e = 1; continue; }
        double dist = norm(sub(ldd(point, q), ldd(point, px)));
        if (fabs(dist - edge_tol) < amb_tol) *amb = 1;
        if (dist > edge_tol) e = 1;
    }
    return e;
}

/* edge [h*w]: the edge pixel rule above applied to one rendered view */
int or_edge_mask(const double *depth, const double *point, int w, int h, double edge_tol, uint8_t *edge) {
    for (int j = 0; j < h; ++j)
        for (int i = 0; i < w; ++i) {
            int amb = 0;
            edge[(int64_t)j * w + i] = (uint8_t)is_edge(depth, point, w, h, i, j, edge_tol, 0.0, &amb);
        }
    return 0;
}

/* the anisotropic colour of one view at image position (u, v) for the texel
 * of face f at surface point p (the readings above).  Two of its decisions
 * are thresholds: the footprint or the centre-sample fallback (UV area at
 * least 1e-4 texel^2), and the tap count N = ceil(s1 / s2 - 0.05).
 * force_centre (-1: decide, 0: footprint, 1: centre sample) and force_taps
 * (0: decide, else that N) fix them.  *amb gets bit0 when the area, bit1 when
 * the ratio lies within rounding of its threshold; *taps the N used. */
static void aniso_core(const float *lv, const int32_t *lf, const float *luv, int W, int H, int32_t f, d3 p,
                       const cam_t *c, const uint8_t *img, const mips_t *m, double u, double v, double lod_bias,
                       int max_taps, int force_centre, int force_taps, double out[3], int *amb, int *taps) {
    double x[3], y[3];
    for (int q = 0; q < 3; ++q) {
        x[q] = (double)luv[6 * (int64_t)f + 2 * q] * W;
        y[q] = (double)luv[6 * (int64_t)f + 2 * q + 1] * H;
    }
    double det = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
    if (fabs(fabs(det) * 0.5 - 1e-4) < 1e-6) *amb |= 1;
    int ok = force_centre < 0 ? fabs(det) * 0.5 >= 1e-4 : !force_centre;
    *taps = 0;
    d3 dpx = mk(0, 0, 0), dpy = mk(0, 0, 0);
    if (ok) {
        double b1x = (y[2] - y[0]) / det, b1y = -(x[2] - x[0]) / det;
        double b2x = -(y[1] - y[0]) / det, b2y = (x[1] - x[0]) / det;
        d3 P0 = ldf(lv, lf[3 * f]), e1 = sub(ldf(lv, lf[3 * f + 1]), P0), e2 = sub(ldf(lv, lf[3 * f + 2]), P0);
        dpx = add(scl(e1, b1x), scl(e2, b2x));
        dpy = add(scl(e1, b1y), scl(e2, b2y));
    }
    double J[2][2];
    for (int a = 0; a < 2 && ok; ++a) {
        d3 dp = a ? dpy : dpx;
        d3 q1 = cam_apply(c, add(p, scl(dp, 0.5))), q0 = cam_apply(c, sub(p, scl(dp, 0.5)));
        if (!(q1.z > 0.0) || !(q0.z > 0.0)) { ok = 0; break; }
        J[0][a] = (c->fx * q1.x / q1.z + c->cx) - (c->fx * q0.x / q0.z + c->cx);
        J[1][a] = (c->fy * q1.y / q1.z + c->cy) - (c->fy * q0.y / q0.z + c->cy);
    }
    if (!ok) {
        for (int ch = 0; ch < 3; ++ch) out[ch] = bilinear(img, m->w[0], m->h[0], ch, u - 0.5, v - 0.5);
        return;
    }
    /* J J^T = [[a, b], [b, d]] */
    double a = J[0][0] * J[0][0] + J[0][1] * J[0][1], b = J[0][0] * J[1][0] + J[0][1] * J[1][1];
    double dd = J[1][0] * J[1][0] + J[1][1] * J[1][1];
    double half = 0.5 * (a + dd), disc = sqrt(0.25 * (a - dd) * (a - dd) + b * b);
    double l1 = half + disc, l2 = half - disc;
    if (l2 < 0.0) l2 = 0.0;
    double s1 = sqrt(l1), s2 = sqrt(l2);
    double ex, ey;
    if (b != 0.0) { ex = l1 - dd; ey = b; }
    else if (a >= dd) { ex = 1.0; ey = 0.0; }
    else { ex = 0.0; ey = 1.0; }
    double en = sqrt(ex * ex + ey * ey);
    ex /= en; ey /= en;
    int N = max_taps;
    if (s2 > 0.0) {
        double ratio = s1 / s2;
        for (int k = 1; k < max_taps; ++k)
            if (fabs(ratio - 0.05 - k) < 1e-4 * ratio) *amb |= 2;
        double nf = ceil(ratio - 0.05);
        N = nf < 1.0 ? 1 : (nf > max_taps ? max_taps : (int)nf);
    }
    if (force_taps > 0) N = force_taps;
    *taps = N;
    double mm = s2 > s1 / max_taps ? s2 : s1 / max_taps;
    double lam = mm > 0.0 ? log2(mm) + lod_bias : 0.0;
    if (lam < 0.0) lam = 0.0;
    if (lam > m->n - 1) lam = m->n - 1;
    for (int ch = 0; ch < 3; ++ch) out[ch] = 0.0;
    for (int i = 0; i < N; ++i) {
        double o = s1 * ((i + 0.5) / N - 0.5);
        for (int ch = 0; ch < 3; ++ch) out[ch] += trilinear(img, m, lam, ch, u + ex * o, v + ey * o);
    }
    for (int ch = 0; ch < 3; ++ch) out[ch] /= N;
}

/* the colour, and where one threshold decision lies within rounding the
 * colour of its other branch: *ncol = 1, 2, or 0 when both decisions are
 * within rounding at once (not enumerated); *fl is set on any of them */
static void aniso_color(const float *lv, const int32_t *lf, const float *luv, int W, int H, int32_t f, d3 p,
                        const cam_t *c, const uint8_t *img, const mips_t *m, double u, double v, double lod_bias,
                        int max_taps, double out[3], double alt[3], int *ncol, uint8_t *fl) {
    int amb = 0, taps = 0;
    aniso_core(lv, lf, luv, W, H, f, p, c, img, m, u, v, lod_bias, max_taps, -1, 0, out, &amb, &taps);
    *ncol = 1;
    if (!amb) return;
    *fl = 1;
    int a2 = 0, t2 = 0;
    if (amb == 1) {
        /* the other side of the area threshold */
        int centre = taps == 0;
        aniso_core(lv, lf, luv, W, H, f, p, c, img, m, u, v, lod_bias, max_taps, !centre, 0, alt, &a2, &t2);
        *ncol = 2;
    } else if (amb == 2 && taps > 0) {
        /* the other side of the tap-count threshold the ratio sits on */
        int lo = taps, hi = taps + 1, other = 0;
        for (int k = 1; k < max_taps; ++k)
            if (k == taps || k + 1 == taps) { lo = k; hi = k + 1; }
        other = taps == hi ? lo : hi;
        if (other < 1) other = 1;
        if (other > max_taps) other = max_taps;
        aniso_core(lv, lf, luv, W, H, f, p, c, img, m, u, v, lod_bias, max_taps, 0, other, alt, &a2, &t2);
        *ncol = other == taps ? 1 : 2;
    } else {
        *ncol = 0;
    }
}

/* the blend of n counted views: sum e^(L_k - m) A_k / (sum e^(L_k - m) + eps e^(-m)), m = max L_k */
static void blend_views(int n, const double *L, double (*A)[3], double eps, double out[3]) {
    double m = L[0];
    for (int k = 1; k < n; ++k) if (L[k] > m) m = L[k];
    double num[3] = {0, 0, 0}, den = 0.0;
    for (int k = 0; k < n; ++k) {
        double e = exp(L[k] - m);
        den += e;
        for (int ch = 0; ch < 3; ++ch) num[ch] += e * A[k][ch];
    }
    den += eps * exp(-m);
    for (int ch = 0; ch < 3; ++ch) out[ch] = num[ch] / den;
}

/* The set of correct results of a flagged texel.  A view is flagged when its
 * inclusion depends on rounding (a pixel or image boundary, a render within
 * rounding, an edge or depth decision within rounding), or, with the
 * anisotropic filter, when its tap count or fallback does; an implementation
 * in another precision may then count the view or not, or take the other
 * branch of the threshold.  Every combination of those choices is a correct
 * result: each view contributes a list of options (absent, and/or present
 * with one of its colours); the blends of all combinations are written,
 * with a filled flag, up to OR_MAX_VARIANTS of them (0 = too many). */
#define OR_MAX_VARIANTS 64
typedef struct { int absent_ok, ncol; double L; double A[2][3]; } view_opt;

static int enumerate_variants(int nv, const view_opt *vo, double eps, double *out /*[OR_MAX_VARIANTS*4]*/) {
    int total = 1;
    for (int k = 0; k < nv; ++k) {
        total *= vo[k].absent_ok + vo[k].ncol;
        if (total > OR_MAX_VARIANTS) return 0;
    }
    for (int c = 0; c < total; ++c) {
        double L[64], A[64][3];
        int n = 0, r = c;
        for (int k = 0; k < nv; ++k) {
            int no = vo[k].absent_ok + vo[k].ncol, o = r % no;
            r /= no;
            if (vo[k].absent_ok && o == 0) continue;
            int col = o - vo[k].absent_ok;
            L[n] = vo[k].L;
            for (int ch = 0; ch < 3; ++ch) A[n][ch] = vo[k].A[col][ch];
            ++n;
        }
        double *dst = out + 4 * (int64_t)c;
        if (n == 0) { dst[0] = dst[1] = dst[2] = 0.0; dst[3] = 0.0; continue; }
        blend_views(n, L, A, eps, dst);
        dst[3] = 1.0;
    }
    return total;
}

/* texture [H*W*3], filled [H*W], flags [H*W], incid (optional) [K*H*W];
 * filter 0: one bilinear sample, 1: anisotropic (the readings above).
 * texels (optional, ntex of them): only these texels (the others are left
 * as they are).  var_* (optional): for up to max_var flagged texels, in
 * order, the texel id, the number of correct results (0: too many to list)
 * and the results [OR_MAX_VARIANTS][rgb, filled]; *n_var the count. */
int or_backproject(const float *lv, int64_t nlv, const int32_t *lf, int64_t nlf, const double *ln, const float *luv,
                   const int32_t *face, const double *bary, int W, int H, int K, const float *cams,
                   const uint8_t *images, int iw, int ih, const double *depth, const double *point, const uint8_t *near,
                   const float *weights, double alpha, double eps, double depth_tol, double edge_tol, double scale,
                   int filter, double lod_bias, int max_taps, double sharpen, double *texture, uint8_t *filled,
                   uint8_t *flags, double *incid, const int64_t *texels, int64_t ntex, int64_t max_var,
                   int64_t *var_tex, uint8_t *var_n, double *var_rgbf, int64_t *n_var) {
    (void)nlv; (void)nlf;
    int64_t npix = (int64_t)iw * ih;
    mips_t *mips = NULL;
    if (n_var) *n_var = 0;
    if (filter) {
        mips = (mips_t *)calloc((size_t)(K > 0 ? K : 1), sizeof(mips_t));
        if (!mips) return -1;
        for (int k = 0; k < K; ++k)
            if (build_mips(images + (int64_t)k * npix * 4, iw, ih, sharpen, &mips[k])) {
                for (int q = 0; q <= k; ++q) free_mips(&mips[q]);
                free(mips);
                return -1;
            }
    }
    int64_t count = texels ? ntex : (int64_t)W * H;
    for (int64_t it = 0; it < count; ++it) {
        int64_t tex = texels ? texels[it] : it;
        texture[3 * tex] = texture[3 * tex + 1] = texture[3 * tex + 2] = 0.0;
        filled[tex] = 0;
        flags[tex] = 0;
        if (incid) for (int k = 0; k < K; ++k) incid[(int64_t)k * W * H + tex] = 0.0;
        int32_t f = face[tex];
        if (f < 0) continue;
        const double *b = bary + 3 * tex;
        d3 p = mk(0, 0, 0), s = mk(0, 0, 0);
        for (int m = 0; m < 3; ++m) {
            p = add(p, scl(ldf(lv, lf[3 * f + m]), b[m]));
            s = add(s, scl(ldd(ln, lf[3 * f + m]), b[m]));
        }
        d3 n = normalize(s);
        double L[64], A[64][3];
        view_opt vo[64];
        int nk = 0, nvo = 0;
        uint8_t fl = 0;
        for (int k = 0; k < K && k < 64; ++k) {
            cam_t c = load_cam(cams + 16 * k);
            d3 q = cam_apply(&c, p);
            if (!(q.z > 0.0)) continue;
            double u = c.fx * q.x / q.z + c.cx, v = c.fy * q.y / q.z + c.cy;
            double fu = u - floor(u), fv = v - floor(v);
            /* ak: whether this view counts depends on rounding */
            int ak = fu < 1e-3 || fu > 1.0 - 1e-3 || fv < 1e-3 || fv > 1.0 - 1e-3;
            int counted = 1;
            if (!(u >= 0.0 && u < iw && v >= 0.0 && v < ih)) {
                counted = 0;
            } else {
                int i = (int)floor(u), j = (int)floor(v);
                const double *dk = depth + (int64_t)k * npix;
                const double *pk = point + (int64_t)k * npix * 3;
                const uint8_t *nk_ = near + (int64_t)k * npix;
                int64_t px = (int64_t)j * iw + i;
                if (nk_[px]) ak = 1;
                {
                    const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
                    for (int nn = 0; nn < 4; ++nn) {
                        int ii = i + di[nn], jj = j + dj[nn];
                        if (ii >= 0 && jj >= 0 && ii < iw && jj < ih && nk_[(int64_t)jj * iw + ii]) ak = 1;
                    }
                }
                if (!(dk[px] < INFINITY)) {
                    counted = 0;
                } else {
                    int amb = 0;
                    int edge = is_edge(dk, pk, iw, ih, i, j, edge_tol, 1e-5 * scale, &amb);
                    if (amb) ak = 1;
                    if (edge) {
                        counted = 0;
                    } else {
                        if (fabs(q.z - (dk[px] + depth_tol)) < 1e-5 * scale) ak = 1;
                        if (q.z > dk[px] + depth_tol) counted = 0;
                    }
                }
            }
            if (ak) fl = 1;
            if (!counted && !ak) continue;
            d3 C = cam_centre(&c);
            double I = dot(n, normalize(sub(C, p)));
            if (!(I > 0.0)) continue;
            double Lk = log((double)weights[k]) + alpha * log(I);
            double col[3], alt[3];
            int ncol = 1;
            if (filter)
                aniso_color(lv, lf, luv, W, H, f, p, &c, images + (int64_t)k * npix * 4, &mips[k], u, v, lod_bias,
                            max_taps, col, alt, &ncol, &fl);
            else
                for (int ch = 0; ch < 3; ++ch)
                    col[ch] = bilinear(images + (int64_t)k * npix * 4, iw, ih, ch, u - 0.5, v - 0.5);
            vo[nvo].absent_ok = ak || !counted;
            vo[nvo].ncol = ncol > 0 ? ncol : 1;
            vo[nvo].L = Lk;
            for (int ch = 0; ch < 3; ++ch) { vo[nvo].A[0][ch] = col[ch]; vo[nvo].A[1][ch] = ncol == 2 ? alt[ch] : col[ch]; }
            if (ncol == 0) vo[nvo].ncol = 99;   /* not enumerable */
            ++nvo;
            if (!counted) continue;
            if (incid) incid[(int64_t)k * W * H + tex] = I;
            L[nk] = log((double)weights[k]) + alpha * log(I);
            for (int ch = 0; ch < 3; ++ch) A[nk][ch] = col[ch];
            ++nk;
        }
        flags[tex] = fl;
        if (fl && var_tex && *n_var < max_var) {
            int64_t j = (*n_var)++;
            var_tex[j] = tex;
            var_n[j] = (uint8_t)enumerate_variants(nvo, vo, eps, var_rgbf + (int64_t)j * OR_MAX_VARIANTS * 4);
        }
        if (nk == 0) continue;
        blend_views(nk, L, A, eps, texture + 3 * tex);
        filled[tex] = 1;
    }
    if (mips) {
        for (int k = 0; k < K; ++k) free_mips(&mips[k]);
        free(mips);
    }
    return 0;
}

/* levels >= 1 of one view's pyramid, unsharpened and sharpened, for pin
 * tests: out [sum of level sizes * 3] per kind; returns the level count */
int or_mip_levels(const uint8_t *img, int w, int h, double sharpen, double *plain, double *sharp, int32_t *dims) {
    mips_t m;
    if (build_mips(img, w, h, sharpen, &m)) return -1;
    size_t off = 0;
    for (int l = 1; l < m.n; ++l) {
        size_t n3 = 3 * (size_t)m.w[l] * m.h[l];
        memcpy(plain + off, m.p[l], n3 * sizeof(double));
        memcpy(sharp + off, m.s[l], n3 * sizeof(double));
        off += n3;
        dims[2 * (l - 1)] = m.w[l];
        dims[2 * (l - 1) + 1] = m.h[l];
    }
    int n = m.n;
    free_mips(&m);
    return n;
}
