/*
 * vsr_oracle.c -- plain CPU reference for custom-intersector ray traversal.
 *
 * TEST INFRASTRUCTURE.  This file is the oracle that the GPU library is
 * checked against.  Only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code, header, table or helper
 * with the CUDA path; it reads the scene arrays, the rays and the serialised
 * BVH blob (whose byte layout it parses itself) and nothing else.
 *
 * What it computes (Zellmann, "Adding Custom Intersectors to the C++ Ray
 * Tracing Template Library Visionaray"):
 *   - intersect(ray, triangle): the paper's FP32 triangle test
 *     (basic_triangle<3, float>, Section 4), taken as Moller-Trumbore (1997)
 *     with the rounding order fixed below;
 *   - intersect(ray, aabb) with the inverse ray direction (Section 4, the
 *     remark after the bvh_costs listing);
 *   - the custom intersector operator() that wraps either test (Section 3.1)
 *     and may clear hr.hit: default (forwards unchanged), alpha texture
 *     (Section 4, alpha-mask listing), procedural alpha (Section 4) and the
 *     bvh_costs counters (Section 4);
 *   - the closest-hit and any-hit queries (Section 3.1) over a linear list of
 *     primitives (brute force) and over a BVH with the while-while traversal
 *     (Section 3.2, after Aila and Laine 2009) in which both calls to
 *     intersect are replaced by the intersector;
 *   - the multi-hit query (the third visibility query of the library the
 *     paper extends, defined in Section 3.1 next to closest-hit and any-hit): the
 *     first N accepted hits in ascending order.  Over a list it is the plain
 *     definition (collect every accepted candidate, sort, keep N); over the
 *     BVH it is the closest-hit traversal with a sorted buffer of N entries
 *     whose last entry plays the role of the closest hit (closest-hit is the
 *     multi-hit query with N = 1);
 *   - instancing (Section 3.2: BVHs acting as compound primitives of a list
 *     or of a top-level BVH, with the intersector passed on to each BVH's own
 *     intersect): an instance is a mesh seen through a world-to-object affine
 *     map W (row-major 3 x 4); the ray is taken to object space as
 *     o'_r = fmaf(W_r0, o.x, fmaf(W_r1, o.y, fmaf(W_r2, o.z, W_r3))),
 *     d'_r = fmaf(W_r0, d.x, fmaf(W_r1, d.y, W_r2 * d.z)), same (tmin, tmax),
 *     so t is the same parameter in both spaces; closest-hit ties between
 *     instances go to the lower instance id, then the lower primitive id.
 *
 * Rounding: compiled with -ffp-contract=off.  Every fused multiply-add is an
 * explicit fmaf(); every other product or sum is a separately rounded FP32
 * operation.  Readings of points the paper leaves open:
 *   - triangle test: e1 = v1 - v0, e2 = v2 - v0, p = d x e2, det = e1.p;
 *     det == 0 is a miss; inv = 1/det; s = o - v0; u = (s.p) inv;
 *     q = s x e1; v = (d.q) inv; t = (e2.q) inv.  Geometric hit iff
 *     u >= 0, v >= 0, u + v <= 1 (closed triangle, both faces);
 *   - dot(a,b) = fmaf(a.x,b.x, fmaf(a.y,b.y, a.z*b.z));
 *     cross(a,b).x = fmaf(a.y,b.z, -(a.z*b.y)) and cyclically;
 *   - a candidate lies strictly inside (tmin, tmax); closest-hit replaces the
 *     current best iff t < t_best or (t == t_best and prim < best prim),
 *     comparing original primitive ids, which makes the answer unique; the
 *     multi-hit order is the same (t, prim) order;
 *   - the intersector is consulted only for geometric candidates inside the
 *     t interval (and, for closest-hit, that would improve the best), which
 *     leaves every hit decision unchanged;
 *   - direction components with |d| < 2^-80 are replaced by +-2^-80 when the
 *     inverse direction is formed; the triangle test uses the original d;
 *   - slab test: t0 = fmaf(lo, invd, -ood), t1 = fmaf(hi, invd, -ood) with
 *     ood = o*invd; tn = max(min(t0,t1) over axes, tmin), tf = min(max(t0,t1)
 *     over axes, t_far); the box is hit iff tn <= tf; t_far is t_best for
 *     closest-hit and tmax for any-hit;
 *   - traversal order: the root box is tested once; at an inner node both
 *     children are tested; if both are hit the child on the side of the ray
 *     direction's sign along the node's split axis is visited first
 *     (left iff the sign bit of d[axis] is clear) and the other is pushed;
 *     stack pops are LIFO with no re-test;
 *   - bvh_costs counts every box test (root included) and every triangle
 *     test, hit or not;
 *   - texture lookup for the alpha decision: nearest texel, clamp to edge,
 *     u -> column, v -> row; 8-bit alpha compared as integers against an
 *     8-bit cutoff, float alpha compared against a float cutoff; primitives
 *     whose texture id is 0xFFFFFFFF are opaque for both alpha intersectors;
 *   - tex-coord interpolation: w0 = (1 - u) - v,
 *     uv = fmaf(v, tc2, fmaf(u, tc1, w0*tc0)) per component;
 *   - procedural alpha: accept iff sinf(f*uv.x) * sinf(f*uv.y) > 0;
 *   - clip box (Section 3.2: an intersector may also replace intersect(ray,
 *     aabb) for the BVH's node boxes): a candidate is accepted iff its hit
 *     point p = fmaf(t, d, o) (per component) lies in the closed clip box; a
 *     node box that does not overlap the clip box counts as missed, and the
 *     far limit of every node box test is also capped at the distance where
 *     the ray leaves the clip box (the slab test above with the clip box, -inf
 *     when the ray misses it).  Neither changes an answer away from hit
 *     points within rounding of a clip face, which are flagged as near ties.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NONE 0xFFFFFFFFu

/* intersector kinds */
enum { ORC_ISECT_NONE = 0, ORC_ISECT_DEFAULT = 1, ORC_ISECT_ALPHA_TEX = 2,
       ORC_ISECT_PROC_ALPHA = 3, ORC_ISECT_COUNT = 4, ORC_ISECT_CLIP = 5 };
/* queries */
enum { ORC_CLOSEST = 0, ORC_ANY = 1, ORC_MULTI = 2 };
/* texture formats */
enum { ORC_TEX_U8 = 0, ORC_TEX_RGBA8 = 1, ORC_TEX_RGBA32F = 2 };
/* near-tie flags */
enum { ORC_TIE_EDGE = 1, ORC_TIE_ALPHA = 2, ORC_TIE_CLIP = 4 };

typedef struct {
    int32_t fmt;
    uint32_t w, h, pad;
    const void* texels;
} orc_texture;

typedef struct {
    const float* verts;      /* [nverts*3] */
    uint64_t nverts;
    const uint32_t* idx;     /* [ntri*3] */
    const float* uvs;        /* [ntri*6]: corner k of prim p at (3p+k)*2 */
    const uint32_t* geom_id; /* [ntri] texture index or ORC_NONE */
    uint32_t ntri, ntex;
    const orc_texture* tex;  /* [ntex] */
} orc_scene;

typedef struct {
    int32_t kind;
    uint32_t cutoff_u8;
    float cutoff_f;
    float freq;
    float clip_lo[3], clip_hi[3]; /* clip-box intersector */
} orc_isect;

typedef struct {
    float o[3], tmin, d[3], tmax;
} orc_ray;

typedef struct {
    float t, u, v;
    uint32_t prim;
} orc_hit;

/* per-ray statistics: box tests, triangle tests, intersector consultations,
 * near-tie flags */
typedef struct {
    uint32_t boxes, tris, cands, flags;
} orc_stats;

/* ------------------------------------------------------------------ */
/* vector helpers with the rounding order fixed                        */

static float dot3(const float a[3], const float b[3]) {
    return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2]));
}

static void cross3(const float a[3], const float b[3], float r[3]) {
    r[0] = fmaf(a[1], b[2], -(a[2] * b[1]));
    r[1] = fmaf(a[2], b[0], -(a[0] * b[2]));
    r[2] = fmaf(a[0], b[1], -(a[1] * b[0]));
}

/* ------------------------------------------------------------------ */
/* intersect(ray, basic_triangle<3,float>) -- geometric test only.    */
/* Returns 1 on a geometric hit; t, u, v are written whenever det!=0. */

static int intersect_triangle(const orc_ray* r, const float v0[3], const float e1[3],
                              const float e2[3], float* t, float* u, float* v) {
    float p[3], s[3], q[3];
    cross3(r->d, e2, p);
    const float det = dot3(e1, p);
    if (det == 0.0f) return -1; /* parallel: no t, u, v */
    const float inv = 1.0f / det;
    s[0] = r->o[0] - v0[0];
    s[1] = r->o[1] - v0[1];
    s[2] = r->o[2] - v0[2];
    *u = dot3(s, p) * inv;
    cross3(s, e1, q);
    *v = dot3(r->d, q) * inv;
    *t = dot3(e2, q) * inv;
    return (*u >= 0.0f && *v >= 0.0f && (*u + *v) <= 1.0f) ? 1 : 0;
}

/* ------------------------------------------------------------------ */
/* Ray set-up shared by the box test: guarded inverse direction.       */

typedef struct {
    orc_ray r;
    float invd[3], ood[3];
} orc_ray_ctx;

static void ray_setup(const orc_ray* in, orc_ray_ctx* c) {
    const float tiny = 0x1p-80f;
    c->r = *in;
    for (int a = 0; a < 3; ++a) {
        float d = in->d[a];
        if (fabsf(d) < tiny) d = copysignf(tiny, d);
        c->invd[a] = 1.0f / d;
        c->ood[a] = in->o[a] * c->invd[a];
    }
}

/* intersect(ray, aabb, inv_dir): slab test against [tmin, t_far]. */
static int intersect_aabb(const orc_ray_ctx* c, const float lo[3], const float hi[3],
                          float t_far) {
    float tn = c->r.tmin, tf = t_far;
    for (int a = 0; a < 3; ++a) {
        const float t0 = fmaf(lo[a], c->invd[a], -c->ood[a]);
        const float t1 = fmaf(hi[a], c->invd[a], -c->ood[a]);
        tn = fmaxf(tn, fminf(t0, t1));
        tf = fminf(tf, fmaxf(t0, t1));
    }
    return tn <= tf;
}

/* ------------------------------------------------------------------ */
/* Texture lookup (nearest, clamp to edge).                            */

static uint32_t texel_index(float c, uint32_t n) {
    const float cl = fminf(fmaxf(c, 0.0f), 1.0f);
    int i = (int)floorf(cl * (float)n);
    if (i > (int)n - 1) i = (int)n - 1;
    return (uint32_t)i;
}

/* alpha decision for texture tx at uv; writes 1 if accepted */
static int alpha_accept(const orc_texture* tx, float x, float y, const orc_isect* is) {
    const uint32_t i = texel_index(x, tx->w), j = texel_index(y, tx->h);
    const uint64_t k = (uint64_t)j * tx->w + i;
    switch (tx->fmt) {
        case ORC_TEX_U8:
            return ((const uint8_t*)tx->texels)[k] >= is->cutoff_u8;
        case ORC_TEX_RGBA8:
            return ((const uint8_t*)tx->texels)[4 * k + 3] >= is->cutoff_u8;
        default:
            return ((const float*)tx->texels)[4 * k + 3] >= is->cutoff_f;
    }
}

/* Interpolated texture coordinate of prim at barycentrics (u, v). */
static void lerp_texcoord(const orc_scene* s, uint32_t prim, float u, float v, float* x,
                          float* y) {
    const float* tc = s->uvs + 6ull * prim;
    const float w0 = (1.0f - u) - v;
    *x = fmaf(v, tc[4], fmaf(u, tc[2], w0 * tc[0]));
    *y = fmaf(v, tc[5], fmaf(u, tc[3], w0 * tc[1]));
}

/* The intersector's verdict on a node box (its intersect(ray, aabb)
 * overload): 0 makes the box count as missed.  Only the clip box culls. */
static int box_keep(const orc_isect* is, const float lo[3], const float hi[3]) {
    if (is->kind != ORC_ISECT_CLIP) return 1;
    for (int a = 0; a < 3; ++a)
        if (lo[a] > is->clip_hi[a] || hi[a] < is->clip_lo[a]) return 0;
    return 1;
}

/* Far limit of node box tests under the intersector: the clip box caps it at
 * the ray's exit distance from the box. */
static float clip_exit(const orc_ray_ctx* c, const orc_isect* is) {
    if (is->kind != ORC_ISECT_CLIP) return INFINITY;
    float tn = -INFINITY, tf = INFINITY;
    for (int a = 0; a < 3; ++a) {
        const float t0 = fmaf(is->clip_lo[a], c->invd[a], -c->ood[a]);
        const float t1 = fmaf(is->clip_hi[a], c->invd[a], -c->ood[a]);
        tn = fmaxf(tn, fminf(t0, t1));
        tf = fminf(tf, fmaxf(t0, t1));
    }
    return tn <= tf ? tf : -INFINITY;
}

/* The intersector's verdict on a geometric candidate at distance t along
 * ray r (the line "hr.hit &= ..." of the user operator()).  Sets near-tie
 * flags. */
static int intersector_accepts(const orc_scene* s, const orc_isect* is, uint32_t prim,
                               float u, float v, const orc_ray* r, float t, uint32_t* flags) {
    if (is->kind == ORC_ISECT_CLIP) {
        int in = 1;
        for (int a = 0; a < 3; ++a) {
            const float p = fmaf(t, r->d[a], r->o[a]);
            in &= p >= is->clip_lo[a] && p <= is->clip_hi[a];
            const double tol = 1e-6 * fmax(1.0, fabs((double)p));
            if (fabs((double)p - is->clip_lo[a]) < tol || fabs((double)p - is->clip_hi[a]) < tol)
                *flags |= ORC_TIE_CLIP;
        }
        return in;
    }
    if (is->kind != ORC_ISECT_ALPHA_TEX && is->kind != ORC_ISECT_PROC_ALPHA) return 1;
    const uint32_t g = s->geom_id[prim];
    if (g == ORC_NONE) return 1;
    float x, y;
    lerp_texcoord(s, prim, u, v, &x, &y);
    if (is->kind == ORC_ISECT_ALPHA_TEX) {
        const orc_texture* tx = &s->tex[g];
        const int a = alpha_accept(tx, x, y, is);
        /* near-tie: the decision changes within 1e-6 of uv */
        const double e = 1e-6;
        const float xs[2] = {(float)((double)x - e), (float)((double)x + e)};
        const float ys[2] = {(float)((double)y - e), (float)((double)y + e)};
        for (int m = 0; m < 2; ++m)
            for (int n = 0; n < 2; ++n)
                if (alpha_accept(tx, xs[m], ys[n], is) != a) *flags |= ORC_TIE_ALPHA;
        return a;
    }
    const float sa = sinf(is->freq * x), sb = sinf(is->freq * y);
    const double exact = sin((double)is->freq * (double)x) * sin((double)is->freq * (double)y);
    if (fabs(exact) < 1e-6) *flags |= ORC_TIE_ALPHA;
    return sa * sb > 0.0f;
}

/* ------------------------------------------------------------------ */
/* Triangle access                                                     */

static void tri_verts(const orc_scene* s, uint32_t prim, float v0[3], float e1[3],
                      float e2[3]) {
    const float* a = s->verts + 3ull * s->idx[3ull * prim];
    const float* b = s->verts + 3ull * s->idx[3ull * prim + 1];
    const float* c = s->verts + 3ull * s->idx[3ull * prim + 2];
    for (int k = 0; k < 3; ++k) {
        v0[k] = a[k];
        e1[k] = b[k] - a[k];
        e2[k] = c[k] - a[k];
    }
}

static void note_edge_tie(float u, float v, uint32_t* flags) {
    double m = (double)u;
    if ((double)v < m) m = v;
    double w = 1.0 - (double)u - (double)v;
    if (w < m) m = w;
    if (fabs(m) < 1e-6) *flags |= ORC_TIE_EDGE;
}

/* (t, prim) comes before hit e in the closest-hit / multi-hit order. */
static int hit_before(float t, uint32_t prim, const orc_hit* e) {
    return t < e->t || (t == e->t && prim < e->prim);
}

/* Insert a hit into the ascending buffer buf[0..nh), dropping its last
 * entry; the caller has checked that the hit comes before that entry. */
static void insert_hit(orc_hit* buf, uint32_t nh, float t, float u, float v, uint32_t prim) {
    uint32_t k = nh - 1;
    while (k > 0 && hit_before(t, prim, &buf[k - 1])) {
        buf[k] = buf[k - 1];
        --k;
    }
    buf[k].t = t;
    buf[k].u = u;
    buf[k].v = v;
    buf[k].prim = prim;
}

/* One primitive tested by the intersector under a query.  Returns 1 when an
 * any-hit query terminates.  `best` holds the running result: one hit for
 * closest-hit and any-hit, the ascending buffer of nh hits for multi-hit
 * (whose last entry bounds the search as the closest hit does). */
static int visit_prim(const orc_scene* s, const orc_isect* is, int query,
                      const orc_ray_ctx* c, uint32_t prim, orc_hit* best, uint32_t nh,
                      orc_stats* st) {
    float v0[3], e1[3], e2[3], t, u, v;
    tri_verts(s, prim, v0, e1, e2);
    st->tris++;
    const int g = intersect_triangle(&c->r, v0, e1, e2, &t, &u, &v);
    if (g < 0) return 0;
    const int in_range = t > c->r.tmin && t < c->r.tmax;
    const orc_hit* last = &best[nh - 1];
    if (in_range) {
        if (query == ORC_ANY || t <= last->t) note_edge_tie(u, v, &st->flags);
    }
    if (g == 0 || !in_range) return 0;
    if (query != ORC_ANY) {
        if (!hit_before(t, prim, last)) return 0;
        st->cands++;
        if (!intersector_accepts(s, is, prim, u, v, &c->r, t, &st->flags)) return 0;
        insert_hit(best, nh, t, u, v, prim);
        return 0;
    }
    st->cands++;
    if (!intersector_accepts(s, is, prim, u, v, &c->r, t, &st->flags)) return 0;
    best->t = t;
    best->u = u;
    best->v = v;
    best->prim = prim;
    return 1;
}

static void miss_record(const orc_ray* r, orc_hit* h) {
    h->t = INFINITY;
    h->u = 0.0f;
    h->v = 0.0f;
    h->prim = ORC_NONE;
    (void)r;
}

/* ------------------------------------------------------------------ */
/* Query over a linear primitive list (no BVH): the intersector        */
/* replaces intersect inside the loop over primitives (Section 3.2).   */

static void list_query(const orc_scene* s, const orc_isect* is, int query,
                       const orc_ray* ray, orc_hit* out, orc_stats* st) {
    orc_ray_ctx c;
    ray_setup(ray, &c);
    orc_hit best;
    best.t = ray->tmax;
    best.u = best.v = 0.0f;
    best.prim = ORC_NONE;
    memset(st, 0, sizeof(*st));
    for (uint32_t p = 0; p < s->ntri; ++p)
        if (visit_prim(s, is, query, &c, p, &best, 1, st)) break;
    if (best.prim == ORC_NONE) miss_record(ray, &best);
    *out = best;
}

static int cmp_hit(const void* a, const void* b) {
    const orc_hit* x = (const orc_hit*)a;
    const orc_hit* y = (const orc_hit*)b;
    if (hit_before(x->t, x->prim, y)) return -1;
    if (hit_before(y->t, y->prim, x)) return 1;
    return 0;
}

/* Multi-hit over the list, as defined: every triangle tested, every
 * geometric candidate inside (tmin, tmax) put to the intersector, the
 * accepted ones sorted by (t, prim) and the first nh kept; missing entries
 * are miss records.  `scratch` holds room for ntri hits. */
static void list_multi(const orc_scene* s, const orc_isect* is, uint32_t nh, const orc_ray* ray,
                       orc_hit* out, orc_hit* scratch, orc_stats* st) {
    orc_ray_ctx c;
    ray_setup(ray, &c);
    memset(st, 0, sizeof(*st));
    uint32_t m = 0;
    for (uint32_t p = 0; p < s->ntri; ++p) {
        float v0[3], e1[3], e2[3], t, u, v;
        tri_verts(s, p, v0, e1, e2);
        st->tris++;
        if (intersect_triangle(&c.r, v0, e1, e2, &t, &u, &v) != 1) continue;
        if (!(t > c.r.tmin && t < c.r.tmax)) continue;
        note_edge_tie(u, v, &st->flags);
        st->cands++;
        if (!intersector_accepts(s, is, p, u, v, &c.r, t, &st->flags)) continue;
        scratch[m].t = t;
        scratch[m].u = u;
        scratch[m].v = v;
        scratch[m].prim = p;
        ++m;
    }
    qsort(scratch, m, sizeof(orc_hit), cmp_hit);
    for (uint32_t k = 0; k < nh; ++k) {
        if (k < m)
            out[k] = scratch[k];
        else
            miss_record(ray, &out[k]);
    }
}

/* ------------------------------------------------------------------ */
/* BVH blob parsing (own reader of the documented byte layout)         */

typedef struct {
    float lo[3];
    uint32_t left_or_first;
    float hi[3];
    uint32_t count_axis;
} orc_node;

typedef struct {
    const orc_node* nodes;
    const uint32_t* order;
    uint32_t num_nodes, num_prims, max_depth;
} orc_bvh;

static int parse_blob(const uint8_t* blob, uint64_t bytes, orc_bvh* b) {
    if (!blob || bytes < 64) return -1;
    if (memcmp(blob, "VSRBVH01", 8) != 0) return -2;
    uint32_t hdr[8];
    memcpy(hdr, blob + 8, sizeof(hdr));
    /* hdr: version, header_bytes, num_nodes, num_prims, max_depth, leaf_max,
     * num_leaves, flags */
    if (hdr[0] != 1 || hdr[1] != 64) return -3;
    b->num_nodes = hdr[2];
    b->num_prims = hdr[3];
    b->max_depth = hdr[4];
    if (bytes != 64ull + 32ull * b->num_nodes + 4ull * b->num_prims) return -4;
    if (b->max_depth > 64 || b->num_nodes < 2) return -5;
    b->nodes = (const orc_node*)(blob + 64);
    b->order = (const uint32_t*)(blob + 64 + 32ull * b->num_nodes);
    return 0;
}

/* ------------------------------------------------------------------ */
/* intersect(ray, BVH): the while-while traversal                      */

/* out: one hit (closest, any) or nh hits in ascending order (multi). */
static void bvh_query(const orc_scene* s, const orc_bvh* b, const orc_isect* is, int query,
                      uint32_t nh, const orc_ray* ray, orc_hit* out, orc_stats* st) {
    orc_ray_ctx c;
    ray_setup(ray, &c);
    orc_hit* best = out;
    if (query != ORC_MULTI) nh = 1;
    for (uint32_t k = 0; k < nh; ++k) {
        best[k].t = ray->tmax;
        best[k].u = best[k].v = 0.0f;
        best[k].prim = ORC_NONE;
    }
    const orc_hit* last = &best[nh - 1];
    memset(st, 0, sizeof(*st));
    uint32_t stack[72];
    int sp = 0;
    if (b->num_prims == 0) goto done;
    const float cap = clip_exit(&c, is);
    st->boxes++;
    if (!intersect_aabb(&c, b->nodes[0].lo, b->nodes[0].hi, fminf(last->t, cap)) ||
        !box_keep(is, b->nodes[0].lo, b->nodes[0].hi))
        goto done;
    uint32_t node = 0;
    for (;;) { /* while ray not terminated */
        while ((b->nodes[node].count_axis >> 2) == 0) { /* while node is inner */
            const orc_node* nd = &b->nodes[node];
            const uint32_t l = nd->left_or_first, r = l + 1;
            const float far_t = fminf((query != ORC_ANY) ? last->t : ray->tmax, cap);
            st->boxes += 2;
            const int hl = intersect_aabb(&c, b->nodes[l].lo, b->nodes[l].hi, far_t) &&
                           box_keep(is, b->nodes[l].lo, b->nodes[l].hi);
            const int hr = intersect_aabb(&c, b->nodes[r].lo, b->nodes[r].hi, far_t) &&
                           box_keep(is, b->nodes[r].lo, b->nodes[r].hi);
            if (hl && hr) {
                const int axis = (int)(nd->count_axis & 3u);
                const int neg = signbit(ray->d[axis]) ? 1 : 0;
                stack[sp++] = neg ? l : r;
                node = neg ? r : l;
            } else if (hl) {
                node = l;
            } else if (hr) {
                node = r;
            } else {
                if (sp == 0) goto done;
                node = stack[--sp];
            }
        }
        /* found a leaf: test its primitives */
        const orc_node* lf = &b->nodes[node];
        const uint32_t first = lf->left_or_first, cnt = lf->count_axis >> 2;
        for (uint32_t k = 0; k < cnt; ++k)
            if (visit_prim(s, is, query, &c, b->order[first + k], best, nh, st)) goto done;
        if (sp == 0) break;
        node = stack[--sp];
    }
done:
    for (uint32_t k = 0; k < nh; ++k)
        if (best[k].prim == ORC_NONE) miss_record(ray, &best[k]);
}

/* ------------------------------------------------------------------ */
/* Instancing: BVHs as compound primitives (Section 3.2)              */

typedef struct {
    float t, u, v;
    uint32_t prim, inst;
} orc_ihit;

typedef struct {
    const orc_scene* scene;
    orc_bvh bvh;
} orc_mesh;

typedef struct {
    const orc_mesh* meshes;
    const uint32_t* inst_mesh; /* [ninst] */
    const float* inst_w2o;     /* [ninst * 12] */
    uint32_t ninst;
    const orc_bvh* top;        /* NULL: the instances form a linear list */
} orc_inst_set;

/* (t, inst, prim) comes before hit e. */
static int ihit_before(float t, uint32_t inst, uint32_t prim, const orc_ihit* e) {
    if (t != e->t) return t < e->t;
    return inst < e->inst || (inst == e->inst && prim < e->prim);
}

static void to_object(const float* w, const orc_ray* r, orc_ray* out) {
    for (int k = 0; k < 3; ++k) {
        const float* m = w + 4 * k;
        out->o[k] = fmaf(m[0], r->o[0], fmaf(m[1], r->o[1], fmaf(m[2], r->o[2], m[3])));
        out->d[k] = fmaf(m[0], r->d[0], fmaf(m[1], r->d[1], m[2] * r->d[2]));
    }
    out->tmin = r->tmin;
    out->tmax = r->tmax;
}

/* One instance: its mesh's while-while traversal with the object-space ray,
 * continuing the running result `best` (the intersector passed on to the
 * mesh's own intersect).  Returns 1 when an any-hit query ends. */
static int instance_query(const orc_mesh* m, const orc_isect* is, int query, uint32_t inst,
                          const orc_ray* obj, orc_ihit* best, orc_stats* st) {
    const orc_bvh* b = &m->bvh;
    const orc_scene* s = m->scene;
    if (b->num_prims == 0) return 0;
    orc_ray_ctx c;
    ray_setup(obj, &c);
    st->boxes++;
    if (!intersect_aabb(&c, b->nodes[0].lo, b->nodes[0].hi,
                        query == ORC_CLOSEST ? best->t : obj->tmax))
        return 0;
    uint32_t stack[72];
    int sp = 0;
    uint32_t node = 0;
    for (;;) {
        while ((b->nodes[node].count_axis >> 2) == 0) {
            const orc_node* nd = &b->nodes[node];
            const uint32_t l = nd->left_or_first, r = l + 1;
            const float far_t = (query == ORC_CLOSEST) ? best->t : obj->tmax;
            st->boxes += 2;
            const int hl = intersect_aabb(&c, b->nodes[l].lo, b->nodes[l].hi, far_t);
            const int hr = intersect_aabb(&c, b->nodes[r].lo, b->nodes[r].hi, far_t);
            if (hl && hr) {
                const int neg = signbit(obj->d[nd->count_axis & 3u]) ? 1 : 0;
                stack[sp++] = neg ? l : r;
                node = neg ? r : l;
            } else if (hl) {
                node = l;
            } else if (hr) {
                node = r;
            } else {
                if (sp == 0) return 0;
                node = stack[--sp];
            }
        }
        const orc_node* lf = &b->nodes[node];
        const uint32_t first = lf->left_or_first, cnt = lf->count_axis >> 2;
        for (uint32_t k = 0; k < cnt; ++k) {
            const uint32_t prim = b->order[first + k];
            float v0[3], e1[3], e2[3], t, u, v;
            tri_verts(s, prim, v0, e1, e2);
            st->tris++;
            const int g = intersect_triangle(&c.r, v0, e1, e2, &t, &u, &v);
            if (g < 0) continue;
            const int in_range = t > c.r.tmin && t < c.r.tmax;
            if (in_range && (query == ORC_ANY || t <= best->t)) note_edge_tie(u, v, &st->flags);
            if (g == 0 || !in_range) continue;
            if (query == ORC_CLOSEST && !ihit_before(t, inst, prim, best)) continue;
            st->cands++;
            if (!intersector_accepts(s, is, prim, u, v, &c.r, t, &st->flags)) continue;
            best->t = t;
            best->u = u;
            best->v = v;
            best->prim = prim;
            best->inst = inst;
            if (query == ORC_ANY) return 1;
        }
        if (sp == 0) return 0;
        node = stack[--sp];
    }
}

/* Closest-hit or any-hit over the instances: a linear list in id order, or
 * the top-level BVH traversed while-while with the world-space ray (the same
 * order rule; its leaves list instance ids). */
static void inst_query(const orc_inst_set* set, const orc_isect* is, int query,
                       const orc_ray* ray, orc_ihit* out, orc_stats* st) {
    orc_ihit best = {ray->tmax, 0.0f, 0.0f, ORC_NONE, ORC_NONE};
    memset(st, 0, sizeof(*st));
    orc_ray obj;
    if (!set->top) {
        for (uint32_t i = 0; i < set->ninst; ++i) {
            to_object(set->inst_w2o + 12ull * i, ray, &obj);
            if (instance_query(&set->meshes[set->inst_mesh[i]], is, query, i, &obj, &best, st))
                break;
        }
    } else if (set->top->num_prims > 0) {
        const orc_bvh* b = set->top;
        orc_ray_ctx c;
        ray_setup(ray, &c);
        st->boxes++;
        if (!intersect_aabb(&c, b->nodes[0].lo, b->nodes[0].hi,
                            query == ORC_CLOSEST ? best.t : ray->tmax))
            goto done;
        uint32_t stack[72];
        int sp = 0;
        uint32_t node = 0;
        for (;;) {
            while ((b->nodes[node].count_axis >> 2) == 0) {
                const orc_node* nd = &b->nodes[node];
                const uint32_t l = nd->left_or_first, r = l + 1;
                const float far_t = (query == ORC_CLOSEST) ? best.t : ray->tmax;
                st->boxes += 2;
                const int hl = intersect_aabb(&c, b->nodes[l].lo, b->nodes[l].hi, far_t);
                const int hr = intersect_aabb(&c, b->nodes[r].lo, b->nodes[r].hi, far_t);
                if (hl && hr) {
                    const int neg = signbit(ray->d[nd->count_axis & 3u]) ? 1 : 0;
                    stack[sp++] = neg ? l : r;
                    node = neg ? r : l;
                } else if (hl) {
                    node = l;
                } else if (hr) {
                    node = r;
                } else {
                    if (sp == 0) goto done;
                    node = stack[--sp];
                }
            }
            const orc_node* lf = &b->nodes[node];
            const uint32_t first = lf->left_or_first, cnt = lf->count_axis >> 2;
            for (uint32_t k = 0; k < cnt; ++k) {
                const uint32_t inst = b->order[first + k];
                to_object(set->inst_w2o + 12ull * inst, ray, &obj);
                if (instance_query(&set->meshes[set->inst_mesh[inst]], is, query, inst, &obj,
                                   &best, st))
                    goto done;
            }
            if (sp == 0) break;
            node = stack[--sp];
        }
    }
done:
    if (best.prim == ORC_NONE) {
        best.t = INFINITY;
        best.u = best.v = 0.0f;
        best.inst = ORC_NONE;
    }
    *out = best;
}

/* ------------------------------------------------------------------ */
/* Threaded drivers                                                    */

typedef struct {
    const orc_scene* s;
    const orc_bvh* b; /* NULL: linear list */
    const orc_isect* is;
    int query;
    uint32_t nh; /* hits per ray (multi-hit), else 1 */
    const orc_ray* rays;
    orc_hit* hits;
    orc_stats* stats;
    uint64_t begin, end;
    const orc_inst_set* set; /* instance queries: hits [n], inst_ids [n] */
    uint32_t* inst_ids;
} orc_job;

static void* run_job(void* arg) {
    orc_job* j = (orc_job*)arg;
    orc_stats tmp;
    orc_hit* scratch = NULL;
    if (!j->b && j->query == ORC_MULTI) {
        scratch = (orc_hit*)malloc(sizeof(orc_hit) * (j->s->ntri ? j->s->ntri : 1));
        if (!scratch) return (void*)1;
    }
    for (uint64_t i = j->begin; i < j->end; ++i) {
        orc_stats* st = j->stats ? &j->stats[i] : &tmp;
        orc_hit* out = &j->hits[i * j->nh];
        if (j->set) {
            orc_ihit h;
            inst_query(j->set, j->is, j->query, &j->rays[i], &h, st);
            out->t = h.t;
            out->u = h.u;
            out->v = h.v;
            out->prim = h.prim;
            if (j->inst_ids) j->inst_ids[i] = h.inst;
        } else if (j->b)
            bvh_query(j->s, j->b, j->is, j->query, j->nh, &j->rays[i], out, st);
        else if (j->query == ORC_MULTI)
            list_multi(j->s, j->is, j->nh, &j->rays[i], out, scratch, st);
        else
            list_query(j->s, j->is, j->query, &j->rays[i], out, st);
    }
    free(scratch);
    return NULL;
}

static int run_threads(orc_job base, uint64_t n, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((uint64_t)nthreads > n) nthreads = n > 0 ? (int)n : 1;
    pthread_t th[256];
    orc_job jobs[256];
    for (int k = 0; k < nthreads; ++k) {
        jobs[k] = base;
        jobs[k].begin = n * (uint64_t)k / (uint64_t)nthreads;
        jobs[k].end = n * (uint64_t)(k + 1) / (uint64_t)nthreads;
    }
    if (nthreads == 1) return run_job(&jobs[0]) ? -7 : 0;
    int started = 0, failed = 0;
    for (int k = 0; k < nthreads; ++k) {
        if (pthread_create(&th[k], NULL, run_job, &jobs[k]) != 0) break;
        ++started;
    }
    for (int k = started; k < nthreads; ++k) failed |= run_job(&jobs[k]) != NULL;
    for (int k = 0; k < started; ++k) {
        void* r = NULL;
        pthread_join(th[k], &r);
        failed |= r != NULL;
    }
    return failed ? -7 : 0;
}

/* ------------------------------------------------------------------ */
/* Exported entry points                                               */

/* Linear-list query (brute force over every triangle). */
int orc_trace_list(const orc_scene* s, const orc_isect* is, int query, const float* rays,
                   uint64_t n, float* hits, uint32_t* stats, int nthreads) {
    if (!s || !is || (n && (!rays || !hits))) return -1;
    if (query != ORC_CLOSEST && query != ORC_ANY) return -1;
    orc_job j = {s, NULL, is, query, 1, (const orc_ray*)rays, (orc_hit*)hits,
                 (orc_stats*)stats, 0, 0, NULL, NULL};
    return run_threads(j, n, nthreads);
}

/* BVH query with the while-while traversal. */
int orc_trace_bvh(const orc_scene* s, const uint8_t* blob, uint64_t bytes,
                  const orc_isect* is, int query, const float* rays, uint64_t n, float* hits,
                  uint32_t* stats, int nthreads) {
    orc_bvh b;
    int rc = parse_blob(blob, bytes, &b);
    if (rc) return rc;
    if (b.num_prims != s->ntri) return -6;
    if (query != ORC_CLOSEST && query != ORC_ANY) return -1;
    orc_job j = {s, &b, is, query, 1, (const orc_ray*)rays, (orc_hit*)hits,
                 (orc_stats*)stats, 0, 0, NULL, NULL};
    return run_threads(j, n, nthreads);
}

/* Multi-hit query: hits [n * nh] (nh per ray, ascending).  blob == NULL:
 * the sorted brute force over the list; otherwise the BVH traversal. */
int orc_trace_multi(const orc_scene* s, const uint8_t* blob, uint64_t bytes,
                    const orc_isect* is, uint32_t nh, const float* rays, uint64_t n,
                    float* hits, uint32_t* stats, int nthreads) {
    if (!s || !is || nh < 1 || (n && (!rays || !hits))) return -1;
    orc_bvh b;
    if (blob) {
        int rc = parse_blob(blob, bytes, &b);
        if (rc) return rc;
        if (b.num_prims != s->ntri) return -6;
    }
    orc_job j = {s, blob ? &b : NULL, is, ORC_MULTI, nh, (const orc_ray*)rays, (orc_hit*)hits,
                 (orc_stats*)stats, 0, 0, NULL, NULL};
    return run_threads(j, n, nthreads);
}

/* Closest-hit / any-hit over instances of meshes (each a scene with its own
 * blob).  top_blob == NULL: the instances form a linear list; otherwise the
 * top-level BVH over them (its primitive i is instance i).  hits [n*4],
 * inst_ids [n] (0xFFFFFFFF on a miss), stats [n*4] or NULL. */
int orc_trace_instances(const orc_scene* const* scenes, const uint8_t* const* blobs,
                        const uint64_t* blob_bytes, uint32_t nmeshes, const uint32_t* inst_mesh,
                        const float* inst_w2o, uint32_t ninst, const uint8_t* top_blob,
                        uint64_t top_bytes, const orc_isect* is, int query, const float* rays,
                        uint64_t n, float* hits, uint32_t* inst_ids, uint32_t* stats,
                        int nthreads) {
    if (!scenes || !blobs || !blob_bytes || !is || (ninst && (!inst_mesh || !inst_w2o)) ||
        (n && (!rays || !hits)))
        return -1;
    if (query != ORC_CLOSEST && query != ORC_ANY) return -1;
    if (is->kind == ORC_ISECT_CLIP) return -1; /* a world-space clip box is not supported */
    orc_mesh* meshes = (orc_mesh*)calloc(nmeshes ? nmeshes : 1, sizeof(orc_mesh));
    if (!meshes) return -7;
    int rc = 0;
    for (uint32_t m = 0; m < nmeshes && rc == 0; ++m) {
        meshes[m].scene = scenes[m];
        rc = parse_blob(blobs[m], blob_bytes[m], &meshes[m].bvh);
        if (rc == 0 && meshes[m].bvh.num_prims != scenes[m]->ntri) rc = -6;
    }
    for (uint32_t i = 0; i < ninst && rc == 0; ++i)
        if (inst_mesh[i] >= nmeshes) rc = -1;
    orc_bvh top;
    if (rc == 0 && top_blob) {
        rc = parse_blob(top_blob, top_bytes, &top);
        if (rc == 0 && top.num_prims != ninst) rc = -6;
    }
    if (rc == 0) {
        orc_inst_set set = {meshes, inst_mesh, inst_w2o, ninst, top_blob ? &top : NULL};
        orc_job j = {NULL, NULL, is, query, 1, (const orc_ray*)rays, (orc_hit*)hits,
                     (orc_stats*)stats, 0, 0, &set, inst_ids};
        rc = run_threads(j, n, nthreads);
    }
    free(meshes);
    return rc;
}

/* Single triangle test, exposed for worked-example checks.  out: t,u,v;
 * returns 1 (hit), 0 (miss) or -1 (parallel). */
int orc_intersect_triangle(const float* ray, const float* v0, const float* v1,
                           const float* v2, float* out) {
    float e1[3], e2[3];
    for (int k = 0; k < 3; ++k) {
        e1[k] = v1[k] - v0[k];
        e2[k] = v2[k] - v0[k];
    }
    return intersect_triangle((const orc_ray*)ray, v0, e1, e2, &out[0], &out[1], &out[2]);
}

/* Single box test with the guarded inverse direction. */
int orc_intersect_aabb(const float* ray, const float* lo, const float* hi, float t_far) {
    orc_ray_ctx c;
    ray_setup((const orc_ray*)ray, &c);
    return intersect_aabb(&c, lo, hi, t_far);
}

/* Shadow rays toward a directional light from primary hit points: origin
 * p = fmaf(t, d, o) per component, direction l, t interval (eps, +inf).  A
 * primary miss gives an inactive ray (tmin 0, tmax -1). */
void orc_shadow_rays(const float* prim_rays, const float* prim_hits, uint64_t n,
                     const float* l, float eps, float* out) {
    for (uint64_t i = 0; i < n; ++i) {
        const orc_ray* r = (const orc_ray*)prim_rays + i;
        const orc_hit* h = (const orc_hit*)prim_hits + i;
        orc_ray* s = (orc_ray*)out + i;
        s->d[0] = l[0];
        s->d[1] = l[1];
        s->d[2] = l[2];
        if (h->prim == ORC_NONE) {
            s->o[0] = s->o[1] = s->o[2] = 0.0f;
            s->tmin = 0.0f;
            s->tmax = -1.0f;
        } else {
            for (int k = 0; k < 3; ++k) s->o[k] = fmaf(h->t, r->d[k], r->o[k]);
            s->tmin = eps;
            s->tmax = INFINITY;
        }
    }
}

/* Ambient-occlusion rays (a workload step, not in the paper): spp rays per
 * primary hit.  Origin fmaf(t, d, o) per component; normal n = normalize of
 * (v1 - v0) x (v2 - v0) turned against the primary direction; tangent frame
 * by the branchless construction of Duff et al. (2017, "Building an
 * orthonormal basis, revisited"); direction for uniforms (x1, x2):
 * sqrt(x1) cos(2 pi x2) t1 + sqrt(x1) sin(2 pi x2) t2 + sqrt(1 - x1) n.  The
 * frame and direction are evaluated in FP64 and rounded to FP32; interval
 * (eps, tmax).  Primary misses give inactive rays (origin 0, direction
 * (0, 0, 1), tmin 0, tmax -1).  Output ray i*spp + k. */
/* ------------------------------------------------------------------ */
/* Path tracing with the intersector: a diffuse path tracer built on    */
/* the closest-hit query (a workload; the paper has no shading).  FP32  */
/* with the operation order fixed so that every bounce is reproducible. */

/* Albedo at a hit: the colour of the nearest texel (the one the alpha
 * decision reads) of a colour texture (RGBA8 / 255, RGBA32F as stored), or
 * `untex` for untextured triangles and alpha-only (u8) textures. */
static void hit_albedo(const orc_scene* s, uint32_t prim, float u, float v, const float untex[3],
                       float out[3]) {
    const uint32_t g = s->geom_id[prim];
    if (g == ORC_NONE || s->tex[g].fmt == ORC_TEX_U8) {
        for (int c = 0; c < 3; ++c) out[c] = untex[c];
        return;
    }
    float x, y;
    lerp_texcoord(s, prim, u, v, &x, &y);
    const orc_texture* tx = &s->tex[g];
    const uint64_t k = (uint64_t)texel_index(y, tx->h) * tx->w + texel_index(x, tx->w);
    for (int c = 0; c < 3; ++c)
        out[c] = tx->fmt == ORC_TEX_RGBA8 ? (float)((const uint8_t*)tx->texels)[4 * k + c] / 255.0f
                                          : ((const float*)tx->texels)[4 * k + c];
}

/* Diffuse bounce from hit h of ray r along the local unit vector l: origin
 * fmaf(t, d, o); face normal m = e1 x e2 (the triangle test's cross),
 * n = m / sqrtf(m . m) (IEEE square root and division; (0, 0, 1) when m = 0),
 * turned against d when n . d > 0; tangent frame of Duff et al. (2017):
 * s = copysignf(1, n.z), a = -1 / (s + n.z), b = (n.x n.y) a,
 * t1 = (1 + ((s n.x) n.x) a, s b, -(s n.x)), t2 = (b, s + (n.y n.y) a, -n.y);
 * direction fmaf(l.x, t1, fmaf(l.y, t2, l.z n)); interval (eps, +inf). */
static void bounce_ray(const orc_scene* s, const orc_ray* r, const orc_hit* h, const float l[3],
                       float eps, orc_ray* out) {
    float v0[3], e1[3], e2[3], m[3], n[3];
    tri_verts(s, h->prim, v0, e1, e2);
    cross3(e1, e2, m);
    const float len = sqrtf(dot3(m, m));
    for (int k = 0; k < 3; ++k) n[k] = len > 0.0f ? m[k] / len : (k == 2 ? 1.0f : 0.0f);
    if (dot3(n, r->d) > 0.0f)
        for (int k = 0; k < 3; ++k) n[k] = -n[k];
    const float sg = copysignf(1.0f, n[2]);
    const float a = -1.0f / (sg + n[2]);
    const float b = (n[0] * n[1]) * a;
    const float sx = sg * n[0];
    const float t1[3] = {1.0f + (sx * n[0]) * a, sg * b, -sx};
    const float t2[3] = {b, sg + (n[1] * n[1]) * a, -n[1]};
    for (int k = 0; k < 3; ++k) {
        out->o[k] = fmaf(h->t, r->d[k], r->o[k]);
        out->d[k] = fmaf(l[0], t1[k], fmaf(l[1], t2[k], l[2] * n[k]));
    }
    out->tmin = eps;
    out->tmax = INFINITY;
}

/* One path: closest hit with the intersector; a miss returns throughput x
 * sky; a hit multiplies the throughput by the albedo and, before `bounces`
 * bounces are spent, continues along dirs[3k..3k+3); after the last bounce's
 * hit the path returns 0. */
static void path_query(const orc_scene* s, const orc_bvh* b, const orc_isect* is,
                       const orc_ray* ray, uint32_t bounces, const float* dirs, float eps,
                       const float sky[3], const float untex[3], float out[3], uint32_t* flags) {
    float f[3] = {1.0f, 1.0f, 1.0f};
    orc_ray cur = *ray;
    out[0] = out[1] = out[2] = 0.0f;
    *flags = 0;
    for (uint32_t k = 0;; ++k) {
        orc_hit h;
        orc_stats st;
        bvh_query(s, b, is, ORC_CLOSEST, 1, &cur, &h, &st);
        *flags |= st.flags;
        if (h.prim == ORC_NONE) {
            for (int c = 0; c < 3; ++c) out[c] = f[c] * sky[c];
            return;
        }
        float alb[3];
        hit_albedo(s, h.prim, h.u, h.v, untex, alb);
        for (int c = 0; c < 3; ++c) f[c] = f[c] * alb[c];
        if (k == bounces) return;
        orc_ray next;
        bounce_ray(s, &cur, &h, dirs + 3ull * k, eps, &next);
        cur = next;
    }
}

typedef struct {
    const orc_scene* s;
    const orc_bvh* b;
    const orc_isect* is;
    const orc_ray* rays;
    uint32_t bounces;
    const float *dirs, *sky, *untex;
    float eps;
    float* radiance;
    uint32_t* flags;
    uint64_t begin, end;
} orc_path_job;

static void* run_path_job(void* arg) {
    orc_path_job* j = (orc_path_job*)arg;
    for (uint64_t i = j->begin; i < j->end; ++i) {
        uint32_t fl;
        path_query(j->s, j->b, j->is, &j->rays[i], j->bounces,
                   j->dirs + 3ull * j->bounces * i, j->eps, j->sky, j->untex,
                   j->radiance + 3 * i, &fl);
        if (j->flags) j->flags[i] = fl;
    }
    return NULL;
}

/* Path tracing over a BVH: radiance [n*3]; dirs [n*bounces*3] local unit
 * vectors (path i's bounce k at 3*(i*bounces + k)); flags [n] the OR of the
 * near-tie flags of every segment, or NULL. */
int orc_path_trace(const orc_scene* s, const uint8_t* blob, uint64_t bytes, const orc_isect* is,
                   const float* rays, uint64_t n, uint32_t bounces, const float* dirs, float eps,
                   const float* sky, const float* untex, float* radiance, uint32_t* flags,
                   int nthreads) {
    if (!s || !is || !sky || !untex || (n && (!rays || !radiance)) ||
        (n && bounces && !dirs))
        return -1;
    orc_bvh b;
    int rc = parse_blob(blob, bytes, &b);
    if (rc) return rc;
    if (b.num_prims != s->ntri) return -6;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((uint64_t)nthreads > n) nthreads = n > 0 ? (int)n : 1;
    pthread_t th[256];
    orc_path_job jobs[256];
    for (int k = 0; k < nthreads; ++k) {
        orc_path_job j = {s, &b, is, (const orc_ray*)rays, bounces, dirs, sky, untex, eps,
                          radiance, flags, n * (uint64_t)k / (uint64_t)nthreads,
                          n * (uint64_t)(k + 1) / (uint64_t)nthreads};
        jobs[k] = j;
    }
    int started = 0;
    for (int k = 1; k < nthreads; ++k) {
        if (pthread_create(&th[k], NULL, run_path_job, &jobs[k]) != 0) break;
        started = k;
    }
    run_path_job(&jobs[0]);
    for (int k = started + 1; k < nthreads; ++k) run_path_job(&jobs[k]);
    for (int k = 1; k <= started; ++k) pthread_join(th[k], NULL);
    return 0;
}

/* One bounce for each of n (ray, hit, local direction) triples: the next
 * segment exactly as the path tracer builds it.  rays/out [n*8], hits [n*4],
 * dirs [n*3]; every hit must name a primitive. */
void orc_bounce(const orc_scene* s, const float* rays, const float* hits, const float* dirs,
                uint64_t n, float eps, float* out) {
    for (uint64_t i = 0; i < n; ++i)
        bounce_ray(s, (const orc_ray*)rays + i, (const orc_hit*)hits + i, dirs + 3 * i, eps,
                   (orc_ray*)out + i);
}

void orc_ao_rays(const orc_scene* s, const float* prim_rays, const float* prim_hits, uint64_t n,
                 uint32_t spp, const float* xi, float tmax, float eps, float* out) {
    for (uint64_t i = 0; i < n; ++i) {
        const orc_ray* r = (const orc_ray*)prim_rays + i;
        const orc_hit* h = (const orc_hit*)prim_hits + i;
        float o[3] = {0.0f, 0.0f, 0.0f};
        double nn[3] = {0.0, 0.0, 1.0};
        const int hit = h->prim != ORC_NONE;
        if (hit) {
            float v0[3], e1[3], e2[3];
            tri_verts(s, h->prim, v0, e1, e2);
            for (int k = 0; k < 3; ++k) o[k] = fmaf(h->t, r->d[k], r->o[k]);
            nn[0] = (double)e1[1] * e2[2] - (double)e1[2] * e2[1];
            nn[1] = (double)e1[2] * e2[0] - (double)e1[0] * e2[2];
            nn[2] = (double)e1[0] * e2[1] - (double)e1[1] * e2[0];
            const double len = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
            for (int k = 0; k < 3; ++k) nn[k] = len > 0 ? nn[k] / len : (k == 2 ? 1.0 : 0.0);
            if (nn[0] * r->d[0] + nn[1] * r->d[1] + nn[2] * r->d[2] > 0)
                for (int k = 0; k < 3; ++k) nn[k] = -nn[k];
        }
        const double sg = copysign(1.0, nn[2]);
        const double a = -1.0 / (sg + nn[2]);
        const double b = nn[0] * nn[1] * a;
        const double t1[3] = {1.0 + sg * nn[0] * nn[0] * a, sg * b, -sg * nn[0]};
        const double t2[3] = {b, sg + nn[1] * nn[1] * a, -nn[1]};
        for (uint32_t k = 0; k < spp; ++k) {
            orc_ray* q = (orc_ray*)out + (i * spp + k);
            if (!hit) {
                q->o[0] = q->o[1] = q->o[2] = 0.0f;
                q->d[0] = q->d[1] = 0.0f;
                q->d[2] = 1.0f;
                q->tmin = 0.0f;
                q->tmax = -1.0f;
                continue;
            }
            const double x1 = xi[2 * (i * spp + k)], x2 = xi[2 * (i * spp + k) + 1];
            const double rr = sqrt(x1), ph = 6.283185307179586 * x2, z = sqrt(1.0 - x1);
            for (int c = 0; c < 3; ++c) {
                q->o[c] = o[c];
                q->d[c] = (float)(rr * cos(ph) * t1[c] + rr * sin(ph) * t2[c] + z * nn[c]);
            }
            q->tmin = eps;
            q->tmax = tmax;
        }
    }
}
