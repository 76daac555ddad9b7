/*
 * Plain FP64 CPU oracle for the SBR channel-modelling hot path of
 * "An SBR Based Ray Tracing Channel Modeling Method for THz and Massive MIMO
 * Communications" (arXiv 2208.10006).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or load
 * this file: only tests/, __graft_entry__.smoke() and the CPU-baseline leg of
 * bench.py use it. It shares no code with the CUDA library.
 *
 * Every step is the slow, obvious form: brute force over all triangles, a
 * direct quadruple loop for H(f), an unblocked Cholesky. FP64 throughout.
 * Where the paper is silent or garbled the reading adopted is stated beside
 * the code; the same readings bind the CUDA path.
 *
 * Steps (paper section / equation):
 *   O1 geodesic launch directions         Sec. II-A.1 (Fig. 1)
 *   O2 trace: closest hit, reception,     Sec. II-A.2, II-A.3
 *      specular bounce
 *   O3 duplicate-path removal             Sec. II-A.2 ("pick out effective paths")
 *   O4 image-method refinement            Sec. I (image method), reading
 *   O5 Fresnel TE/TM x roughness          Sec. II-B.1, Eq. 6-8
 *   O6 spreading + atmosphere             Eq. 1, 3, 9, 10
 *   O7 MIMO H(f), near-field delays       Sec. II-C, Eq. 11-14
 *   O8 PDP, path loss, RMS delay spread,  Eq. 2, 4, 5, Table I quantities
 *      mean AoD/AoA
 *   O9 capacity                           Eq. 15-17 (garbled; reading stated)
 *
 * Parity unpinned (no closed form, only self-consistency): the alpha
 * definition (maximum adjacent-ray angle), which candidate ray a duplicate key
 * keeps, the capacity normalisation reading and the arithmetic-mean angles.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_KMAX 8
#define ORC_C0 299792458.0
#define ORC_EPS0 8.8541878128e-12
#define ORC_PI 3.14159265358979323846

/* edge-ambiguity flag bits (per ray) */
#define ORC_FLAG_NEAR_EDGE 1
#define ORC_FLAG_T_TIE 2
#define ORC_FLAG_RADIUS 4
#define ORC_FLAG_TSTAR 8
#define ORC_FLAG_GRAZING 16

typedef struct { double x, y, z; } v3;

static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double norm(v3 a) { return sqrt(dot(a, a)); }
static v3 unit(v3 a) { return scl(a, 1.0 / norm(a)); }
static v3 ld3(const double* p) { return mk(p[0], p[1], p[2]); }
static void st3(double* p, v3 a) { p[0] = a.x; p[1] = a.y; p[2] = a.z; }
static double minf(double a, double b) { return a < b ? a : b; }

/* ------------------------------------------------------------------------ */
/* O1: icosahedron ray launching (Sec. II-A.1, Fig. 1).                       */
/* Reading: class-I frequency-N subdivision of each icosahedron face, flat    */
/* then projected to the unit sphere. Ray order: the 12 vertices; then per    */
/* edge (sorted pairs a<b at distance 2) the N-1 interior edge points; then  */
/* per face (sorted triples) the interior points i>=1, j>=1, i+j<=N-1 with i  */
/* outer. Count 10N^2+2.                                                      */
/* ------------------------------------------------------------------------ */

static void ico_vertices(double V[12][3]) {
    const double ph = (1.0 + sqrt(5.0)) / 2.0;
    const double sg[4][2] = {{1, 1}, {1, -1}, {-1, 1}, {-1, -1}};
    for (int k = 0; k < 4; ++k) {
        V[k][0] = 0;              V[k][1] = sg[k][0];        V[k][2] = sg[k][1] * ph;
        V[4 + k][0] = sg[k][0];   V[4 + k][1] = sg[k][1] * ph; V[4 + k][2] = 0;
        V[8 + k][0] = sg[k][0] * ph; V[8 + k][1] = 0;        V[8 + k][2] = sg[k][1];
    }
}

static int ico_is_edge(double V[12][3], int a, int b) {
    double dx = V[a][0] - V[b][0], dy = V[a][1] - V[b][1], dz = V[a][2] - V[b][2];
    return fabs(dx * dx + dy * dy + dz * dz - 4.0) < 1e-9;
}

/* edges[30][2], faces[20][3], both in lexicographic order */
static void ico_topology(double V[12][3], int edges[30][2], int faces[20][3]) {
    int ne = 0, nf = 0;
    for (int a = 0; a < 12; ++a)
        for (int b = a + 1; b < 12; ++b)
            if (ico_is_edge(V, a, b)) { edges[ne][0] = a; edges[ne][1] = b; ++ne; }
    for (int a = 0; a < 12; ++a)
        for (int b = a + 1; b < 12; ++b)
            for (int c = b + 1; c < 12; ++c)
                if (ico_is_edge(V, a, b) && ico_is_edge(V, b, c) && ico_is_edge(V, a, c)) {
                    faces[nf][0] = a; faces[nf][1] = b; faces[nf][2] = c; ++nf;
                }
}

int64_t orc_geodesic_count(int32_t N) { return 10 * (int64_t)N * N + 2; }

/* Directions of rays [r0, r1) in enumeration order into out[(r1-r0)*3].
 * Returns the total count R, or -1 if N < 1. */
static int64_t geodesic_range(int32_t N, int64_t r0, int64_t r1, double* out) {
    if (N < 1) return -1;
    double V[12][3]; int E[30][2], Fc[20][3];
    ico_vertices(V); ico_topology(V, E, Fc);
    int64_t r = 0;
#define ORC_EMIT(expr) do { if (r >= r0 && r < r1) st3(out + 3 * (r - r0), unit(expr)); ++r; } while (0)
    for (int k = 0; k < 12; ++k) ORC_EMIT(ld3(V[k]));
    for (int e = 0; e < 30; ++e) {
        v3 a = ld3(V[E[e][0]]), b = ld3(V[E[e][1]]);
        for (int k = 1; k <= N - 1; ++k) ORC_EMIT(add(a, scl(sub(b, a), (double)k / N)));
    }
    for (int f = 0; f < 20; ++f) {
        v3 a = ld3(V[Fc[f][0]]), b = ld3(V[Fc[f][1]]), c = ld3(V[Fc[f][2]]);
        for (int i = 1; i <= N - 2; ++i)
            for (int j = 1; i + j <= N - 1; ++j)
                ORC_EMIT(add(a, add(scl(sub(b, a), (double)i / N), scl(sub(c, a), (double)j / N))));
    }
#undef ORC_EMIT
    return r;
}

/* out[R*3]; returns R, or -1 if N < 1 */
int64_t orc_geodesic_dirs(int32_t N, double* out) {
    return geodesic_range(N, 0, orc_geodesic_count(N), out);
}

static double angle_between(v3 a, v3 b) { return atan2(norm(cross(a, b)), dot(a, b)); }

/* alpha (Sec. II-A.3 reception-sphere radius needs the angular ray spacing).
 * Reading: the largest angle between two directions joined by an edge of
 * the subdivided icosahedron's sub-triangles. */
double orc_geodesic_alpha(int32_t N) {
    static int32_t cached_N = 0;
    static double cached = 0.0;
    if (N < 1) return -1.0;
    if (N == cached_N) return cached;
    double V[12][3]; int E[30][2], Fc[20][3];
    ico_vertices(V); ico_topology(V, E, Fc);
    double best = 0.0;
    for (int f = 0; f < 20; ++f) {
        v3 a = ld3(V[Fc[f][0]]), b = ld3(V[Fc[f][1]]), c = ld3(V[Fc[f][2]]);
        for (int i = 0; i < N; ++i)
            for (int j = 0; i + j < N; ++j) {
                v3 p00 = unit(add(a, add(scl(sub(b, a), (double)i / N), scl(sub(c, a), (double)j / N))));
                v3 p10 = unit(add(a, add(scl(sub(b, a), (double)(i + 1) / N), scl(sub(c, a), (double)j / N))));
                v3 p01 = unit(add(a, add(scl(sub(b, a), (double)i / N), scl(sub(c, a), (double)(j + 1) / N))));
                double t1 = angle_between(p00, p10), t2 = angle_between(p00, p01),
                       t3 = angle_between(p10, p01);
                if (t1 > best) best = t1;
                if (t2 > best) best = t2;
                if (t3 > best) best = t3;
            }
    }
    cached_N = N;
    cached = best;
    return best;
}

/* ------------------------------------------------------------------------ */
/* scene                                                                      */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t T;
    int32_t S;
    v3 (*v)[3];    /* FP64 copies of the FP32 vertices */
    v3* n;         /* unit normal of each triangle */
    const int32_t* surf;
    /* per surface: its triangles in ascending face id (CSR) */
    int64_t* s_off;
    int64_t* s_tri;
} scene_t;

static int scene_init(scene_t* sc, const float* tri, const int32_t* surf, int64_t T, int32_t S) {
    memset(sc, 0, sizeof *sc);
    sc->T = T; sc->S = S; sc->surf = surf;
    sc->v = malloc(sizeof(v3[3]) * (T > 0 ? T : 1));
    sc->n = malloc(sizeof(v3) * (T > 0 ? T : 1));
    sc->s_off = calloc((size_t)S + 1, sizeof(int64_t));
    sc->s_tri = malloc(sizeof(int64_t) * (T > 0 ? T : 1));
    if (!sc->v || !sc->n || !sc->s_off || !sc->s_tri) return -1;
    for (int64_t t = 0; t < T; ++t) {
        for (int k = 0; k < 3; ++k)
            sc->v[t][k] = mk(tri[9 * t + 3 * k], tri[9 * t + 3 * k + 1], tri[9 * t + 3 * k + 2]);
        sc->n[t] = unit(cross(sub(sc->v[t][1], sc->v[t][0]), sub(sc->v[t][2], sc->v[t][0])));
        if (surf[t] < 0 || surf[t] >= S) return -2;
        sc->s_off[surf[t] + 1]++;
    }
    for (int s = 0; s < S; ++s) sc->s_off[s + 1] += sc->s_off[s];
    int64_t* fill = calloc((size_t)S, sizeof(int64_t));
    for (int64_t t = 0; t < T; ++t) sc->s_tri[sc->s_off[surf[t]] + fill[surf[t]]++] = t;
    free(fill);
    return 0;
}

static void scene_free(scene_t* sc) {
    free(sc->v); free(sc->n); free(sc->s_off); free(sc->s_tri);
}

/* plane of a surface: that of its lowest-id triangle (reading) */
static int surface_plane(const scene_t* sc, int s, v3* n, double* c) {
    if (s < 0 || s >= sc->S || sc->s_off[s] == sc->s_off[s + 1]) return -1;
    int64_t t = sc->s_tri[sc->s_off[s]];
    *n = sc->n[t];
    *c = dot(*n, sc->v[t][0]);
    return 0;
}

/* Moller-Trumbore in FP64. Returns 0 if the ray is parallel to the plane;
 * else t and barycentrics (u, v, w=1-u-v) of the line/plane intersection. */
static int mt(v3 o, v3 d, const v3* tv, double* t, double* u, double* v) {
    v3 e1 = sub(tv[1], tv[0]), e2 = sub(tv[2], tv[0]);
    v3 p = cross(d, e2);
    double det = dot(e1, p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    v3 s = sub(o, tv[0]);
    *u = dot(s, p) * inv;
    v3 q = cross(s, e1);
    *v = dot(d, q) * inv;
    *t = dot(e2, q) * inv;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* O2: trace (Sec. II-A.2 ray tracing, Sec. II-A.3 reception).                */
/* Readings: rays start at the Tx reference point; surfaces are two-sided;   */
/* the segment after a reflection ignores every face of the surface just     */
/* hit; the nearest hit is the smallest t > 0, ties to the lowest face id;   */
/* no power threshold: rays run to K reflections or escape. For b = 0..K the */
/* segment is tested against every receiver: t* = (Rx-o).d, received if      */
/* 0 <= t* <= t_hit and |o + t* d - Rx| <= alpha (L + t*) / sqrt(3), L the    */
/* unfolded length before the segment (ray-cone cross-section).               */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t rx, nb;
    int32_t seq[ORC_KMAX];
    int64_t ray;
    double dist;
    int32_t flags;
    int32_t pad;
} orc_cand;

typedef struct {
    int64_t rays, segments, flagged_rays;
} orc_trace_counters;

typedef struct {
    const scene_t* sc;
    v3 tx;
    const double* rx; int32_t n_rx;
    int32_t N, K; double alpha, eps;
    const double* dirs; /* directions of rays [dir_base, ...) */
    int64_t dir_base;
    int64_t r0, r1;
    orc_cand* buf; int64_t n, cap;
    uint8_t* flags; /* [r1 - r0], relative to the global ray_begin */
    int64_t flag_base;
    int64_t segments, flagged;
    int oom;
} trace_job;

static void push_cand(trace_job* j, orc_cand* c) {
    if (j->n == j->cap) {
        int64_t nc = j->cap ? 2 * j->cap : 256;
        orc_cand* nb = realloc(j->buf, sizeof(orc_cand) * nc);
        if (!nb) { j->oom = 1; return; }
        j->buf = nb; j->cap = nc;
    }
    j->buf[j->n++] = *c;
}

/* closest hit over all triangles except those of surface `skip`.
 * Returns the face id (or -1) and t_hit (INFINITY when none). */
static int64_t closest_hit(const scene_t* sc, v3 o, v3 d, int skip, double* t_hit) {
    int64_t best = -1; double bt = INFINITY;
    for (int64_t t = 0; t < sc->T; ++t) {
        if (sc->surf[t] == skip) continue;
        double tt, u, v;
        if (!mt(o, d, sc->v[t], &tt, &u, &v)) continue;
        double w = 1.0 - u - v;
        if (u >= 0 && v >= 0 && w >= 0 && tt > 0) {
            if (tt < bt || (tt == bt && t < best)) { bt = tt; best = t; }
        }
    }
    *t_hit = bt;
    return best;
}

/* Edge-ambiguity of one segment: a different outcome lies within eps
 * (relative) of this one. Flags: the hit triangle's barycentric margin is
 * within eps; a triangle of another surface in front is missed or hit within
 * eps of its edge; two surfaces are hit within eps relative in t; the ray is
 * nearly parallel to a face it could hit. */
static int segment_flags(const scene_t* sc, v3 o, v3 d, int skip, int64_t best, double bt,
                         double eps) {
    int fl = 0;
    int bs = best >= 0 ? sc->surf[best] : -1;
    double lim = isinf(bt) ? INFINITY : bt * (1.0 + eps);
    for (int64_t t = 0; t < sc->T; ++t) {
        if (sc->surf[t] == skip) continue;
        double tt, u, v;
        v3 e1 = sub(sc->v[t][1], sc->v[t][0]), e2 = sub(sc->v[t][2], sc->v[t][0]);
        double det = dot(e1, cross(d, e2));
        double sc_ = norm(e1) * norm(e2);
        if (fabs(det) <= eps * sc_) {
            /* nearly parallel: flag if the plane is met in front, close to the triangle */
            if (mt(o, d, sc->v[t], &tt, &u, &v) && tt > 0 && tt <= lim) {
                double m = minf(minf(u, v), 1.0 - u - v);
                if (m >= -eps) fl |= ORC_FLAG_GRAZING;
            }
            continue;
        }
        if (!mt(o, d, sc->v[t], &tt, &u, &v)) continue;
        if (!(tt > 0 && tt <= lim)) continue;
        double m = minf(minf(u, v), 1.0 - u - v);
        if (t == best) {
            if (m <= eps) fl |= ORC_FLAG_NEAR_EDGE;
        } else if (sc->surf[t] != bs) {
            if (fabs(m) <= eps) fl |= ORC_FLAG_NEAR_EDGE;
            if (m >= 0 && best >= 0 && fabs(tt - bt) <= eps * bt) fl |= ORC_FLAG_T_TIE;
        }
    }
    return fl;
}

static void trace_ray(trace_job* j, int64_t ray) {
    const scene_t* sc = j->sc;
    v3 o = j->tx, d = ld3(j->dirs + 3 * (ray - j->dir_base));
    double L = 0.0;
    int prev = -1, nb = 0;
    int32_t seq[ORC_KMAX];
    int flags = 0;
    const double inv_sqrt3 = 1.0 / sqrt(3.0);
    for (int b = 0; b <= j->K; ++b) {
        double bt;
        int64_t best = closest_hit(sc, o, d, prev, &bt);
        flags |= segment_flags(sc, o, d, prev, best, bt, j->eps);
        j->segments++;
        /* reception (Sec. II-A.3) */
        for (int r = 0; r < j->n_rx; ++r) {
            v3 R = ld3(j->rx + 3 * r);
            double ts = dot(sub(R, o), d);
            double s = L + ts;
            v3 p = add(o, scl(d, ts));
            double dist = norm(sub(p, R));
            double rad = j->alpha * s * inv_sqrt3;
            if (ts >= 0 && ts <= bt && dist <= rad) {
                orc_cand c;
                memset(&c, 0, sizeof c);
                c.rx = r; c.nb = nb;
                for (int k = 0; k < ORC_KMAX; ++k) c.seq[k] = k < nb ? seq[k] : -1;
                c.ray = ray; c.dist = dist;
                push_cand(j, &c);
            }
            /* boundary of the reception decision */
            if (dist <= rad * (1.0 + j->eps) + 0.0 && ts >= -j->eps * fabs(s) &&
                ts <= bt + j->eps * fabs(s)) {
                if (fabs(dist - rad) <= j->eps * rad) flags |= ORC_FLAG_RADIUS;
                if (fabs(ts) <= j->eps * fabs(s) || (!isinf(bt) && fabs(ts - bt) <= j->eps * fabs(s)))
                    flags |= ORC_FLAG_TSTAR;
            }
        }
        if (b == j->K || best < 0) break;
        /* specular bounce: d' = d - 2 (d.n) n on the hit face's plane */
        o = add(o, scl(d, bt));
        v3 n = sc->n[best];
        d = sub(d, scl(n, 2.0 * dot(d, n)));
        L += bt;
        prev = sc->surf[best];
        seq[nb++] = prev;
    }
    if (flags) {
        j->flagged++;
        for (int64_t c = j->n - 1; c >= 0 && j->buf[c].ray == ray; --c) j->buf[c].flags = flags;
    }
    j->flags[ray - j->flag_base] = (uint8_t)flags;
}

static void* trace_worker(void* arg) {
    trace_job* j = arg;
    for (int64_t r = j->r0; r < j->r1; ++r) trace_ray(j, r);
    return NULL;
}

/*
 * Trace rays [ray_begin, ray_end) of the geodesic set for subdivision N.
 * tri: FP32 [T*9]; surf: [T] in [0,S); tx: [3]; rx: [n_rx*3].
 * Candidates are returned through *out (malloc'd, release with orc_free) in
 * ray order; ray_flags[ray_end-ray_begin] receives the edge-ambiguity bits.
 * Returns the number of candidates, or a negative error.
 */
int64_t orc_trace(const float* tri, const int32_t* surf, int64_t T, int32_t S,
                  const double* tx, const double* rx, int32_t n_rx, int32_t N, int32_t K,
                  double alpha, int64_t ray_begin, int64_t ray_end, double eps,
                  int32_t nthreads, orc_cand** out, uint8_t* ray_flags,
                  orc_trace_counters* counters) {
    if (N < 1 || K < 0 || K > ORC_KMAX || ray_begin < 0 || ray_end < ray_begin) return -1;
    int64_t R = orc_geodesic_count(N);
    if (ray_end > R) return -1;
    scene_t sc;
    if (scene_init(&sc, tri, surf, T, S) != 0) { scene_free(&sc); return -2; }
    int64_t nr_all = ray_end - ray_begin;
    double* dirs = malloc(sizeof(double) * 3 * (nr_all > 0 ? nr_all : 1));
    if (!dirs) { scene_free(&sc); return -3; }
    geodesic_range(N, ray_begin, ray_end, dirs);
    if (alpha <= 0) alpha = orc_geodesic_alpha(N);
    if (nthreads < 1) nthreads = 1;
    int64_t nr = ray_end - ray_begin;
    if (nthreads > nr) nthreads = nr > 0 ? (int32_t)nr : 1;
    trace_job* jobs = calloc((size_t)nthreads, sizeof(trace_job));
    pthread_t* th = calloc((size_t)nthreads, sizeof(pthread_t));
    for (int i = 0; i < nthreads; ++i) {
        trace_job* j = &jobs[i];
        j->sc = &sc; j->tx = ld3(tx); j->rx = rx; j->n_rx = n_rx; j->N = N; j->K = K;
        j->alpha = alpha; j->eps = eps; j->dirs = dirs; j->dir_base = ray_begin;
        j->r0 = ray_begin + nr * i / nthreads; j->r1 = ray_begin + nr * (i + 1) / nthreads;
        j->flags = ray_flags; j->flag_base = ray_begin;
        pthread_create(&th[i], NULL, trace_worker, j);
    }
    int64_t total = 0; int oom = 0;
    orc_trace_counters cnt = {nr, 0, 0};
    for (int i = 0; i < nthreads; ++i) {
        pthread_join(th[i], NULL);
        total += jobs[i].n; oom |= jobs[i].oom;
        cnt.segments += jobs[i].segments; cnt.flagged_rays += jobs[i].flagged;
    }
    orc_cand* all = malloc(sizeof(orc_cand) * (total > 0 ? total : 1));
    int64_t at = 0;
    for (int i = 0; i < nthreads; ++i) {
        if (jobs[i].n) memcpy(all + at, jobs[i].buf, sizeof(orc_cand) * jobs[i].n);
        at += jobs[i].n;
        free(jobs[i].buf);
    }
    free(jobs); free(th); free(dirs); scene_free(&sc);
    if (counters) *counters = cnt;
    if (oom || !all) { free(all); return -3; }
    *out = all;
    return total;
}

void orc_free(void* p) { free(p); }

/*
 * Per-segment record of one ray, for sampled checks against another
 * implementation: seg_o[(K+1)*3] origins, seg_face[K+1] hit face (-1 = escape),
 * seg_t[K+1] t_hit. Returns the number of segments traced.
 */
int32_t orc_trace_one(const float* tri, const int32_t* surf, int64_t T, int32_t S,
                      const double* tx, int32_t N, int32_t K, int64_t ray, double* seg_o,
                      double* seg_d, int64_t* seg_face, double* seg_t, double* seg_L) {
    if (N < 1 || K < 0 || K > ORC_KMAX || ray < 0 || ray >= orc_geodesic_count(N)) return -1;
    scene_t sc;
    if (scene_init(&sc, tri, surf, T, S) != 0) { scene_free(&sc); return -2; }
    double dir[3];
    geodesic_range(N, ray, ray + 1, dir);
    v3 o = ld3(tx), d = ld3(dir);
    double L = 0; int prev = -1; int32_t ns = 0;
    for (int b = 0; b <= K; ++b) {
        double bt;
        int64_t best = closest_hit(&sc, o, d, prev, &bt);
        st3(seg_o + 3 * b, o); st3(seg_d + 3 * b, d);
        seg_face[b] = best; seg_t[b] = bt; seg_L[b] = L; ns++;
        if (b == K || best < 0) break;
        o = add(o, scl(d, bt));
        v3 n = sc.n[best];
        d = sub(d, scl(n, 2.0 * dot(d, n)));
        L += bt; prev = sc.surf[best];
    }
    scene_free(&sc);
    return ns;
}

/* ------------------------------------------------------------------------ */
/* O3: duplicate-path removal (Sec. II-A.2 "pick out effective paths").       */
/* Reading: key = (rx, sequence of surface ids); a planar specular surface   */
/* sequence defines at most one physical path. Kept: minimum dist, ties to   */
/* the lower ray id. all_flagged = every candidate of the key came from an    */
/* edge-ambiguous ray.                                                        */
/* ------------------------------------------------------------------------ */

static int key_cmp(const orc_cand* a, const orc_cand* b) {
    if (a->rx != b->rx) return a->rx < b->rx ? -1 : 1;
    if (a->nb != b->nb) return a->nb < b->nb ? -1 : 1;
    for (int k = 0; k < a->nb; ++k)
        if (a->seq[k] != b->seq[k]) return a->seq[k] < b->seq[k] ? -1 : 1;
    return 0;
}

static int cand_cmp(const void* pa, const void* pb) {
    const orc_cand* a = pa; const orc_cand* b = pb;
    int c = key_cmp(a, b);
    if (c) return c;
    if (a->dist != b->dist) return a->dist < b->dist ? -1 : 1;
    if (a->ray != b->ray) return a->ray < b->ray ? -1 : 1;
    return 0;
}

/* Sorts cands in place; writes one record per key into keys (capacity n) in
 * (rx, nb, seq) order; n_prod[k] = candidates of that key; all_flagged[k].
 * Returns the number of keys. */
int64_t orc_dedup(orc_cand* cands, int64_t n, orc_cand* keys, int64_t* n_prod,
                  int32_t* all_flagged) {
    if (n <= 0) return 0;
    qsort(cands, (size_t)n, sizeof(orc_cand), cand_cmp);
    int64_t nk = 0;
    for (int64_t i = 0; i < n;) {
        int64_t j = i;
        int allf = 1;
        while (j < n && key_cmp(&cands[i], &cands[j]) == 0) {
            if (!cands[j].flags) allf = 0;
            ++j;
        }
        keys[nk] = cands[i];
        n_prod[nk] = j - i;
        all_flagged[nk] = allf;
        ++nk;
        i = j;
    }
    return nk;
}

/* ------------------------------------------------------------------------ */
/* O4: image-method refinement of a surface sequence (reading; the paper     */
/* names the image method in Sec. I). Mirror the Tx through the planes in    */
/* order, back-trace from the Rx, require every intersection parameter in    */
/* (0,1) and every point inside one of its surface's triangles (barycentric  */
/* tolerance 1e-9); report the lowest-id such triangle. L = |I_m - Rx|.      */
/* No occlusion recheck: the ray already demonstrated visibility.            */
/* ------------------------------------------------------------------------ */

static int point_in_tri(const v3* tv, v3 p, double tol) {
    v3 e1 = sub(tv[1], tv[0]), e2 = sub(tv[2], tv[0]), w = sub(p, tv[0]);
    double d00 = dot(e1, e1), d01 = dot(e1, e2), d11 = dot(e2, e2);
    double d20 = dot(w, e1), d21 = dot(w, e2);
    double den = d00 * d11 - d01 * d01;
    if (den == 0.0) return 0;
    double b1 = (d11 * d20 - d01 * d21) / den;
    double b2 = (d00 * d21 - d01 * d20) / den;
    double b0 = 1.0 - b1 - b2;
    return b0 >= -tol && b1 >= -tol && b2 >= -tol;
}

static void angles_deg(v3 v, double* az, double* el) {
    *az = atan2(v.y, v.x) * 180.0 / ORC_PI;
    *el = atan2(v.z, hypot(v.x, v.y)) * 180.0 / ORC_PI;
}

/*
 * For each key: valid[p], face[p*KMAX], pts[p*KMAX*3], L[p], aod[p*2], aoa[p*2].
 * Returns the number of valid paths.
 */
int64_t orc_refine(const float* tri, const int32_t* surf, int64_t T, int32_t S,
                   const double* tx, const double* rx, const orc_cand* keys, int64_t n,
                   int32_t* valid, int32_t* face, double* pts, double* L, double* aod,
                   double* aoa) {
    scene_t sc;
    if (scene_init(&sc, tri, surf, T, S) != 0) { scene_free(&sc); return -2; }
    v3 Tx = ld3(tx);
    int64_t nv = 0;
    for (int64_t p = 0; p < n; ++p) {
        const orc_cand* k = &keys[p];
        v3 Rx = ld3(rx + 3 * k->rx);
        int m = k->nb;
        int ok = 1;
        v3 img[ORC_KMAX + 1], P[ORC_KMAX + 1], nn[ORC_KMAX + 1];
        double cc[ORC_KMAX + 1];
        for (int i = 0; i < ORC_KMAX; ++i) {
            face[p * ORC_KMAX + i] = -1;
            st3(pts + (p * ORC_KMAX + i) * 3, mk(0, 0, 0));
        }
        img[0] = Tx;
        for (int i = 1; i <= m && ok; ++i) {
            if (surface_plane(&sc, k->seq[i - 1], &nn[i], &cc[i]) != 0) { ok = 0; break; }
            img[i] = sub(img[i - 1], scl(nn[i], 2.0 * (dot(nn[i], img[i - 1]) - cc[i])));
        }
        v3 target = Rx;
        for (int i = m; i >= 1 && ok; --i) {
            v3 dv = sub(target, img[i]);
            double den = dot(nn[i], dv);
            if (den == 0.0) { ok = 0; break; }
            double u = (cc[i] - dot(nn[i], img[i])) / den;
            if (!(u > 0.0 && u < 1.0)) { ok = 0; break; }
            P[i] = add(img[i], scl(dv, u));
            target = P[i];
        }
        for (int i = 1; i <= m && ok; ++i) {
            int s = k->seq[i - 1];
            int64_t found = -1;
            for (int64_t q = sc.s_off[s]; q < sc.s_off[s + 1]; ++q) {
                int64_t t = sc.s_tri[q];
                if (point_in_tri(sc.v[t], P[i], 1e-9)) { found = t; break; }
            }
            if (found < 0) { ok = 0; break; }
            face[p * ORC_KMAX + i - 1] = (int32_t)found;
            st3(pts + (p * ORC_KMAX + i - 1) * 3, P[i]);
        }
        valid[p] = ok;
        if (!ok) { L[p] = NAN; continue; }
        ++nv;
        L[p] = norm(sub(img[m], Rx));
        v3 first = m ? P[1] : Rx, last = m ? P[m] : Tx;
        angles_deg(sub(first, Tx), &aod[2 * p], &aod[2 * p + 1]);
        angles_deg(sub(last, Rx), &aoa[2 * p], &aoa[2 * p + 1]);
    }
    scene_free(&sc);
    return nv;
}

/* ------------------------------------------------------------------------ */
/* O5 + O6: complex path gain g_n(f).                                         */
/* Eq. 6-8: rho = exp(-g/2), g = (4 pi sigma_h cos(theta_i) / lambda)^2,      */
/* r' = rho r_TE/TM. The Fresnel formula is not printed (Sec. II-B.1);        */
/* reading: lossy dielectric eta = eps_r - j sigma/(2 pi f eps0),             */
/* Gamma_TE = (cos - sqrt(eta - sin^2)) / (cos + sqrt(eta - sin^2)),          */
/* Gamma_TM = (eta cos - sqrt(eta - sin^2)) / (eta cos + sqrt(eta - sin^2)).  */
/* Polarimetric tracking (reading of Eq. 1): E0 = pol(d0); per bounce         */
/* s = unit(d_in x n), p_in = s x d_in, p_out = s x d_out,                    */
/* E <- rho [Gamma_TE (E.s) s + Gamma_TM (E.p_in) p_out]; Rx projection       */
/* pol(d_last).E. Eq. 3 with beta = 1 and unit Tx power gives the Friis       */
/* amplitude c/(4 pi f L); Eq. 9 gives 10^(-gamma L / 20000) (gamma in dB/km,  */
/* L in m); Eq. 10 adds the phase -phi (pi/180) L / 1000. The delay phasor    */
/* exp(-j 2 pi f L / c) is not part of g.                                     */
/* ------------------------------------------------------------------------ */

typedef double complex cplx;

static v3 pol_vec(v3 d, int pol) {
    double th = atan2(hypot(d.x, d.y), d.z);  /* polar angle */
    double ph = atan2(d.y, d.x);
    if (pol == 0) return mk(cos(th) * cos(ph), cos(th) * sin(ph), -sin(th)); /* V: theta-hat */
    return mk(-sin(ph), cos(ph), 0.0);                                      /* H: phi-hat */
}

void orc_fresnel(double eps_r, double sigma, double f, double cos_i, double* te_re,
                 double* te_im, double* tm_re, double* tm_im) {
    cplx eta = eps_r - I * sigma / (2.0 * ORC_PI * f * ORC_EPS0);
    double s2 = 1.0 - cos_i * cos_i;
    cplx root = csqrt(eta - s2);
    cplx te = (cos_i - root) / (cos_i + root);
    cplx tm = (eta * cos_i - root) / (eta * cos_i + root);
    *te_re = creal(te); *te_im = cimag(te); *tm_re = creal(tm); *tm_im = cimag(tm);
}

double orc_roughness(double rough_m, double f, double cos_i) {
    double g = 4.0 * ORC_PI * rough_m * cos_i * f / ORC_C0;
    return exp(-0.5 * g * g);
}

/* per-axis choice when d_in is parallel to n: s = unit(n x e), e the axis of
 * the smallest |n| component (first on ties) */
static v3 s_vector(v3 din, v3 n) {
    v3 cr = cross(din, n);
    double l = norm(cr);
    if (l > 1e-12) return scl(cr, 1.0 / l);
    v3 e = mk(1, 0, 0);
    double ax = fabs(n.x), ay = fabs(n.y), az = fabs(n.z);
    if (ay < ax && ay <= az) e = mk(0, 1, 0);
    else if (az < ax && az < ay) e = mk(0, 0, 1);
    return unit(cross(n, e));
}

/*
 * g[p*F + f] (complex128 interleaved) for every path. Paths as written by
 * orc_refine (only valid ones are passed). mats[S*3] = eps_r, sigma, rough.
 * pol: 0 = V (theta-hat), 1 = H (phi-hat).
 */
int32_t orc_gains(const float* tri, const int32_t* surf, int64_t T, int32_t S, const double* mats,
                  const double* tx, const double* rx, int64_t P, const int32_t* rxi,
                  const int32_t* nb, const int32_t* seq, const double* pts, const double* L,
                  const double* freqs, int32_t F, const double* gamma_db_km,
                  const double* disp_deg_km, int32_t pol, double* g) {
    scene_t sc;
    if (scene_init(&sc, tri, surf, T, S) != 0) { scene_free(&sc); return -2; }
    for (int64_t p = 0; p < P; ++p) {
        int m = nb[p];
        v3 pt[ORC_KMAX + 2];
        pt[0] = ld3(tx);
        for (int i = 1; i <= m; ++i) pt[i] = ld3(pts + (p * ORC_KMAX + i - 1) * 3);
        pt[m + 1] = ld3(rx + 3 * rxi[p]);
        for (int32_t fi = 0; fi < F; ++fi) {
            double f = freqs[fi];
            v3 d0 = unit(sub(pt[1], pt[0]));
            v3 e0 = pol_vec(d0, pol);
            cplx E[3] = {e0.x, e0.y, e0.z};
            for (int i = 1; i <= m; ++i) {
                int s = seq[p * ORC_KMAX + i - 1];
                v3 n; double c;
                surface_plane(&sc, s, &n, &c);
                v3 din = unit(sub(pt[i], pt[i - 1]));
                v3 dout = unit(sub(pt[i + 1], pt[i]));
                double cos_i = fabs(dot(din, n));
                double tr, ti, mr, mi;
                orc_fresnel(mats[3 * s], mats[3 * s + 1], f, cos_i, &tr, &ti, &mr, &mi);
                double rho = orc_roughness(mats[3 * s + 2], f, cos_i);
                cplx gte = rho * (tr + I * ti), gtm = rho * (mr + I * mi);
                v3 sv = s_vector(din, n);
                v3 pin = cross(sv, din), pout = cross(sv, dout);
                cplx es = E[0] * sv.x + E[1] * sv.y + E[2] * sv.z;
                cplx ep = E[0] * pin.x + E[1] * pin.y + E[2] * pin.z;
                E[0] = gte * es * sv.x + gtm * ep * pout.x;
                E[1] = gte * es * sv.y + gtm * ep * pout.y;
                E[2] = gte * es * sv.z + gtm * ep * pout.z;
            }
            v3 dl = unit(sub(pt[m + 1], pt[m]));
            v3 pr = pol_vec(dl, pol);
            cplx proj = pr.x * E[0] + pr.y * E[1] + pr.z * E[2];
            double amp = ORC_C0 / (4.0 * ORC_PI * f * L[p]);
            double att = pow(10.0, -gamma_db_km[fi] * L[p] / 20000.0);
            double ph = -disp_deg_km[fi] * (ORC_PI / 180.0) * L[p] / 1000.0;
            cplx v = amp * att * cexp(I * ph) * proj;
            g[2 * (p * F + fi)] = creal(v);
            g[2 * (p * F + fi) + 1] = cimag(v);
        }
    }
    scene_free(&sc);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* O7: H(f) for one receiver reference point (Eq. 11-14; near field,          */
/* Sec. I). Reading: amplitudes and coefficients from the reference geometry; */
/* phase from exact per-element spherical distances with fixed interaction    */
/* points. For a reflected path n with first/last points P1/Pm:               */
/*   dt_pn = |T_p - P1| - |T_0 - P1|,  dr_qn = |R_q - Pm| - |R_0 - Pm|,        */
/*   H[f,q,p] += g_n(f) exp(-j 2 pi f (L_n + dt_pn + dr_qn) / c).              */
/* A LoS path uses the exact |T_p - R_q| in its phase. Direct quadruple loop; */
/* the phase is reduced as frac(f L / c) in FP64.                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t f0, f1;
    int32_t F, Nt, Nr; int64_t P;
    const double *freqs, *tx_elem, *rx_elem, *pts, *L, *g;
    const int32_t* nb;
    v3 T0, R0;
    double* H;
} synth_job;

static void* synth_worker(void* arg) {
    synth_job* j = arg;
    for (int64_t fi = j->f0; fi < j->f1; ++fi) {
        double f = j->freqs[fi];
        for (int32_t q = 0; q < j->Nr; ++q) {
            v3 Rq = ld3(j->rx_elem + 3 * q);
            for (int32_t p = 0; p < j->Nt; ++p) {
                v3 Tp = ld3(j->tx_elem + 3 * p);
                double hr = 0, hi = 0;
                for (int64_t n = 0; n < j->P; ++n) {
                    int m = j->nb[n];
                    double len;
                    if (m == 0) {
                        len = norm(sub(Tp, Rq));
                    } else {
                        v3 P1 = ld3(j->pts + (n * ORC_KMAX) * 3);
                        v3 Pm = ld3(j->pts + (n * ORC_KMAX + m - 1) * 3);
                        double dt = norm(sub(Tp, P1)) - norm(sub(j->T0, P1));
                        double dr = norm(sub(Rq, Pm)) - norm(sub(j->R0, Pm));
                        len = j->L[n] + dt + dr;
                    }
                    double cyc = f * len / ORC_C0;
                    double fr = cyc - floor(cyc);
                    double ang = -2.0 * ORC_PI * fr;
                    double gr = j->g[2 * (n * j->F + fi)], gi = j->g[2 * (n * j->F + fi) + 1];
                    double c = cos(ang), s = sin(ang);
                    hr += gr * c - gi * s;
                    hi += gr * s + gi * c;
                }
                j->H[2 * ((fi * j->Nr + q) * (int64_t)j->Nt + p)] = hr;
                j->H[2 * ((fi * j->Nr + q) * (int64_t)j->Nt + p) + 1] = hi;
            }
        }
    }
    return NULL;
}

/* H[F*Nr*Nt] complex128 interleaved. Paths are those of one receiver. */
int32_t orc_synth_H(int64_t P, const int32_t* nb, const double* pts, const double* L,
                    const double* g, const double* freqs, int32_t F, const double* tx_ref,
                    const double* rx_ref, const double* tx_elem, int32_t Nt,
                    const double* rx_elem, int32_t Nr, int32_t nthreads, double* H) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > F) nthreads = F > 0 ? F : 1;
    synth_job* jobs = calloc((size_t)nthreads, sizeof(synth_job));
    pthread_t* th = calloc((size_t)nthreads, sizeof(pthread_t));
    for (int i = 0; i < nthreads; ++i) {
        synth_job* j = &jobs[i];
        j->f0 = (int64_t)F * i / nthreads; j->f1 = (int64_t)F * (i + 1) / nthreads;
        j->F = F; j->Nt = Nt; j->Nr = Nr; j->P = P;
        j->freqs = freqs; j->tx_elem = tx_elem; j->rx_elem = rx_elem; j->pts = pts; j->L = L;
        j->g = g; j->nb = nb; j->T0 = ld3(tx_ref); j->R0 = ld3(rx_ref); j->H = H;
        pthread_create(&th[i], NULL, synth_worker, j);
    }
    for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
    free(jobs); free(th);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Per-element reception (Sec. I near field, Eq. 13-14, Fig. 11): every       */
/* receive element q is traced as a receiver of its own, and its H row sums   */
/* its own paths. Paths n of element q (rx[n] == q) with unfolded length L_n: */
/*   H[f,q,p] = sum_n g_n(f) exp(-j 2 pi f len_np / c),                       */
/*   len_np = |T_p - R_q| for the LoS path,                                   */
/*   len_np = L_n + |T_p - P1| - |T_0 - P1| otherwise (P1 the first point);   */
/* the Rx side needs no correction because R_q is the traced receiver.        */
/* ------------------------------------------------------------------------ */

int32_t orc_synth_H_elements(int64_t P, const int32_t* rx, const int32_t* nb, const double* pts,
                             const double* L, const double* g, const double* freqs, int32_t F,
                             const double* tx_ref, const double* tx_elem, int32_t Nt,
                             const double* rx_elem, int32_t Nr, double* H) {
    v3 T0 = ld3(tx_ref);
    for (int64_t i = 0; i < (int64_t)F * Nr * Nt * 2; ++i) H[i] = 0.0;
    for (int64_t n = 0; n < P; ++n) {
        int32_t q = rx[n];
        if (q < 0 || q >= Nr) return -1;
        v3 Rq = ld3(rx_elem + 3 * q);
        int m = nb[n];
        for (int32_t p = 0; p < Nt; ++p) {
            v3 Tp = ld3(tx_elem + 3 * p);
            double len;
            if (m == 0) {
                len = norm(sub(Tp, Rq));
            } else {
                v3 P1 = ld3(pts + (n * ORC_KMAX) * 3);
                double dt = norm(sub(Tp, P1)) - norm(sub(T0, P1));
                len = L[n] + dt;
            }
            for (int32_t fi = 0; fi < F; ++fi) {
                double cyc = freqs[fi] * len / ORC_C0;
                double ang = -2.0 * ORC_PI * (cyc - floor(cyc));
                double gr = g[2 * (n * F + fi)], gi = g[2 * (n * F + fi) + 1];
                double c = cos(ang), s = sin(ang);
                int64_t o = 2 * ((fi * (int64_t)Nr + q) * Nt + p);
                H[o] += gr * c - gi * s;
                H[o + 1] += gr * s + gi * c;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* O8: PDP and channel statistics of one receiver (Eq. 2, 4, 5; Table I).     */
/* Reading: absolute delay tau = L / c, bins [k, k+1) * bin_s; tap = sum of   */
/* |g_n(f_c)|^2 falling in the bin, in dB (empty bins -inf). PL_inc =         */
/* -10 log10 sum |g|^2; PL_coh = -10 log10 |sum g exp(-j 2 pi f_c tau)|^2     */
/* (Eq. 2); tau_rms per Eq. 5 with P_n = |g_n|^2; mean AoD/AoA: power-        */
/* weighted arithmetic means of azimuth and elevation (degrees).              */
/* stats[7] = PL_coh, PL_inc, tau_rms, aod_az, aod_el, aoa_az, aoa_el.        */
/* ------------------------------------------------------------------------ */

int32_t orc_pdp_stats(int64_t P, const double* L, const double* g_fc /*complex [P]*/,
                      const double* aod, const double* aoa, double fc, double bin_s,
                      int32_t n_bins, double* pdp_db, double* stats) {
    double* acc = calloc((size_t)(n_bins > 0 ? n_bins : 1), sizeof(double));
    double sp = 0, st = 0, st2 = 0, cr = 0, ci = 0;
    double a1 = 0, a2 = 0, a3 = 0, a4 = 0;
    for (int64_t n = 0; n < P; ++n) {
        double gr = g_fc[2 * n], gi = g_fc[2 * n + 1];
        double pw = gr * gr + gi * gi;
        double tau = L[n] / ORC_C0;
        double kb = floor(tau / bin_s);
        if (kb >= 0 && kb < n_bins) acc[(int64_t)kb] += pw;
        sp += pw; st += pw * tau; st2 += pw * tau * tau;
        double cyc = fc * L[n] / ORC_C0;
        double ang = -2.0 * ORC_PI * (cyc - floor(cyc));
        cr += gr * cos(ang) - gi * sin(ang);
        ci += gr * sin(ang) + gi * cos(ang);
        a1 += pw * aod[2 * n]; a2 += pw * aod[2 * n + 1];
        a3 += pw * aoa[2 * n]; a4 += pw * aoa[2 * n + 1];
    }
    for (int32_t k = 0; k < n_bins; ++k) pdp_db[k] = acc[k] > 0 ? 10.0 * log10(acc[k]) : -INFINITY;
    free(acc);
    if (P == 0 || sp <= 0) {
        stats[0] = stats[1] = INFINITY;
        for (int k = 2; k < 7; ++k) stats[k] = NAN;
        return 0;
    }
    stats[0] = -10.0 * log10(cr * cr + ci * ci);
    stats[1] = -10.0 * log10(sp);
    double m1 = st / sp, m2 = st2 / sp;
    double var = m2 - m1 * m1;
    stats[2] = sqrt(var > 0 ? var : 0.0);
    stats[3] = a1 / sp; stats[4] = a2 / sp; stats[5] = a3 / sp; stats[6] = a4 / sp;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* O9: capacity (Eq. 15-17). Eq. 16 multiplies by Q = sum |h|^2, which taken  */
/* literally drives C to ~0 at realistic path loss; reading: Frobenius        */
/* normalisation W_f = (Nr Nt / Qbar) H_f H_f^H (H^H H when Nt < Nr), Qbar =  */
/* mean over f of ||H_f||_F^2; n = min(Nr, Nt); SNR linear 10^(dB/10);        */
/* C = mean_f log2 det(I_n + SNR/Nt W_f) by an FP64 complex Cholesky.         */
/* ------------------------------------------------------------------------ */

static double logdet_hpd(cplx* A, int n) {
    /* in-place lower Cholesky; returns ln det or NAN if not positive definite */
    double ld = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = creal(A[j * n + j]);
        for (int k = 0; k < j; ++k) d -= creal(A[j * n + k] * conj(A[j * n + k]));
        if (!(d > 0)) return NAN;
        double ljj = sqrt(d);
        A[j * n + j] = ljj;
        ld += 2.0 * log(ljj);
        for (int i = j + 1; i < n; ++i) {
            cplx s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= A[i * n + k] * conj(A[j * n + k]);
            A[i * n + j] = s / ljj;
        }
    }
    return ld;
}

/* H: complex128 interleaved [F*Nr*Nt]; C_out[n_snr] */
int32_t orc_capacity(const double* H, int32_t F, int32_t Nr, int32_t Nt, const double* snr_db,
                     int32_t n_snr, double* C_out) {
    if (F < 1 || Nr < 1 || Nt < 1) return -1;
    const cplx* h = (const cplx*)H;
    double q = 0;
    for (int64_t i = 0; i < (int64_t)F * Nr * Nt; ++i) q += creal(h[i] * conj(h[i]));
    q /= F;
    if (!(q > 0)) { for (int s = 0; s < n_snr; ++s) C_out[s] = 0.0; return 0; }
    int n = Nr < Nt ? Nr : Nt;
    cplx* W = malloc(sizeof(cplx) * n * n);
    cplx* A = malloc(sizeof(cplx) * n * n);
    for (int s = 0; s < n_snr; ++s) C_out[s] = 0.0;
    for (int32_t f = 0; f < F; ++f) {
        const cplx* Hf = h + (int64_t)f * Nr * Nt;
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) {
                cplx acc = 0;
                if (Nt >= Nr) { /* (H H^H)[a,b] = sum_p H[a,p] conj(H[b,p]) */
                    for (int p = 0; p < Nt; ++p) acc += Hf[a * Nt + p] * conj(Hf[b * Nt + p]);
                } else {        /* (H^H H)[a,b] = sum_q conj(H[q,a]) H[q,b] */
                    for (int qq = 0; qq < Nr; ++qq) acc += conj(Hf[qq * Nt + a]) * Hf[qq * Nt + b];
                }
                W[a * n + b] = acc * ((double)Nr * Nt / q);
            }
        for (int s = 0; s < n_snr; ++s) {
            double snr = pow(10.0, snr_db[s] / 10.0);
            for (int a = 0; a < n; ++a)
                for (int b = 0; b < n; ++b)
                    A[a * n + b] = (a == b ? 1.0 : 0.0) + (snr / Nt) * W[a * n + b];
            C_out[s] += logdet_hpd(A, n) / log(2.0);
        }
    }
    for (int s = 0; s < n_snr; ++s) C_out[s] /= F;
    free(W); free(A);
    return 0;
}
