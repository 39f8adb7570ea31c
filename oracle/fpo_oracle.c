/*
 * FP64 CPU oracle for Fourier PlenOctree (FPO) rendering.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library; both read the same seeded
 * inputs and nothing else.
 *
 * What it computes, in the paper's order (Wang et al., "Fourier PlenOctrees
 * for Dynamic Radiance Field Rendering in Real-time", CVPR 2022):
 *   - the real Fourier basis IDFT_i(t) of Eq. 8 (Sec. 4.1);
 *   - density sigma(t) = sum_{i<n1} k^sigma_i IDFT_i(t) (Eq. 7), clamped at 0
 *     (the paper prints no activation; max(0, .) is this build's reading);
 *   - SH coefficients z_{m,l}(t) = sum_{i<n2} k^z_{m,l,i} IDFT_i(t) (Eq. 9),
 *     with i in [0, n2-1];
 *   - colour c(d) = S(sum_{l,m} z_{m,l} Y_{m,l}(d)) with S the sigmoid (Eq. 1),
 *     real SH of degree <= 2 in closed form (sign convention: the real part /
 *     imaginary part of the complex SH with the Condon-Shortley phase,
 *     times sqrt 2);
 *   - emission-absorption compositing over the exact ray-leaf segments of the
 *     union octree (Sec. 4.2 union structure; PlenOctree-style volume
 *     rendering, Sec. 3): alpha = 1 - exp(-sigma delta), C += T alpha c,
 *     T *= 1 - alpha, stop once T < stop_T (tested after each update), then
 *     C += T bg.
 *
 * Segments are found by plain recursion over the tree: every leaf box is
 * slab-tested in FP64, every leaf with t_out - t_in > 0 (t clipped at 0) is
 * kept, and the list is sorted by entry distance.  No DDA, no stepping.
 *
 * Near-tie flags (per ray): bit 0 is set when some leaf box has
 * |t_out - t_in| <= 1e-6 (the ray grazes an edge or corner, so an FP32
 * traversal may legitimately visit or skip it), or a zero direction
 * component lies within 1e-6 of a box plane; bit 1 is set when ln T comes
 * within 1e-3 of ln stop_T after some update (an FP32 renderer may stop one
 * step earlier or later).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-2)
#define ORC_ERR_TREE (-4)

#define NEAR_FACE_EPS 1e-6
#define NEAR_STOP_LOG_EPS 1e-3

/* ------------------------------------------------------------------------ */
/* Eq. 8: IDFT_i(t) = cos(i pi t / T) for even i, sin((i+1) pi t / T) for odd i */
int oracle_basis(int n, double t, double period, double *out)
{
    if (n < 0 || period <= 0.0 || !out) return ORC_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        if (i % 2 == 0)
            out[i] = cos((double)i * M_PI * t / period);
        else
            out[i] = sin((double)(i + 1) * M_PI * t / period);
    }
    return ORC_OK;
}

/* Eq. 1: real SH Y_{m,l}(d) for l <= degree (<= 2), index k = l(l+1)+m,
 * d a unit vector (x, y, z). */
int oracle_sh(int degree, const double *d, double *out)
{
    if (degree < 0 || degree > 2 || !d || !out) return ORC_ERR_ARG;
    const double x = d[0], y = d[1], z = d[2];
    out[0] = 0.5 * sqrt(1.0 / M_PI);
    if (degree >= 1) {
        const double c1 = sqrt(3.0 / (4.0 * M_PI));
        out[1] = -c1 * y;
        out[2] = c1 * z;
        out[3] = -c1 * x;
    }
    if (degree >= 2) {
        const double c2 = 0.5 * sqrt(15.0 / M_PI);
        out[4] = c2 * x * y;
        out[5] = -c2 * y * z;
        out[6] = 0.25 * sqrt(5.0 / M_PI) * (3.0 * z * z - 1.0);
        out[7] = -c2 * x * z;
        out[8] = 0.25 * sqrt(15.0 / M_PI) * (x * x - y * y);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Union octree as a plain pointer-free node pool built by inserting leaves. */
typedef struct {
    int32_t child[8]; /* node index or -1; octant = 4*bx + 2*by + bz */
    int32_t leaf;     /* leaf id (upload order) or -1 */
} onode;

typedef struct {
    onode *nodes;
    int32_t n_nodes, cap;
    int32_t n_leaves, max_depth;
} otree;

static int32_t node_new(otree *tr)
{
    if (tr->n_nodes == tr->cap) {
        int32_t nc = tr->cap ? tr->cap * 2 : 1024;
        onode *nn = (onode *)realloc(tr->nodes, (size_t)nc * sizeof(onode));
        if (!nn) return -1;
        tr->nodes = nn;
        tr->cap = nc;
    }
    onode *n = &tr->nodes[tr->n_nodes];
    for (int i = 0; i < 8; ++i) n->child[i] = -1;
    n->leaf = -1;
    return tr->n_nodes++;
}

void oracle_tree_free(void *p)
{
    otree *tr = (otree *)p;
    if (!tr) return;
    free(tr->nodes);
    free(tr);
}

/* Builds the tree from leaf cells; *status = ORC_ERR_TREE when a leaf lies
 * outside its level's grid, duplicates another, or contains/is contained in
 * another leaf (union-tree leaves are disjoint, Sec. 4.2). */
void *oracle_tree_new(int32_t n_leaves, int32_t max_depth, const uint8_t *leaf_depth,
                      const uint32_t *leaf_xyz, int *status)
{
    *status = ORC_ERR_ARG;
    if (n_leaves < 0 || max_depth < 0 || max_depth > 20) return NULL;
    if (n_leaves > 0 && (!leaf_depth || !leaf_xyz)) return NULL;
    otree *tr = (otree *)calloc(1, sizeof(otree));
    if (!tr) { *status = ORC_ERR_OOM; return NULL; }
    tr->n_leaves = n_leaves;
    tr->max_depth = max_depth;
    if (node_new(tr) < 0) { oracle_tree_free(tr); *status = ORC_ERR_OOM; return NULL; }
    for (int32_t id = 0; id < n_leaves; ++id) {
        int dep = leaf_depth[id];
        uint32_t x = leaf_xyz[3 * id], y = leaf_xyz[3 * id + 1], z = leaf_xyz[3 * id + 2];
        if (dep > max_depth || (x >> dep) || (y >> dep) || (z >> dep)) {
            oracle_tree_free(tr); *status = ORC_ERR_TREE; return NULL;
        }
        int32_t cur = 0;
        for (int l = 0; l < dep; ++l) {
            if (tr->nodes[cur].leaf >= 0) { oracle_tree_free(tr); *status = ORC_ERR_TREE; return NULL; }
            int s = dep - 1 - l;
            int oct = 4 * ((x >> s) & 1) + 2 * ((y >> s) & 1) + ((z >> s) & 1);
            int32_t nx = tr->nodes[cur].child[oct];
            if (nx < 0) {
                nx = node_new(tr);
                if (nx < 0) { oracle_tree_free(tr); *status = ORC_ERR_OOM; return NULL; }
                tr->nodes[cur].child[oct] = nx;
            }
            cur = nx;
        }
        onode *n = &tr->nodes[cur];
        int has_child = 0;
        for (int i = 0; i < 8; ++i) has_child |= (n->child[i] >= 0);
        if (n->leaf >= 0 || has_child) { oracle_tree_free(tr); *status = ORC_ERR_TREE; return NULL; }
        n->leaf = id;
    }
    *status = ORC_OK;
    return tr;
}

/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t n1, n2, sh_degree;
    double period_T;
    const float *coeffs; /* [n_leaves][n1 + 3*(deg+1)^2*n2], canonical order */
    double aabb_min[3];
    double aabb_size;
    double bg[3];
    double stop_T;
} oracle_scene;

typedef struct {
    int32_t mode; /* 0: pinhole camera, 1: explicit rays */
    double eye[3], target[3], up[3];
    double fov_y_deg;
    int32_t width, height;
    double t; /* frame time for camera mode, and for ray mode when t_per_ray is NULL */
    int64_t n;                 /* ray mode: number of rays */
    const double *o, *d;       /* ray mode: [n][3]; d need not be unit */
    const double *t_per_ray;   /* ray mode, optional [n] */
    int64_t n_sel;             /* optional subset of ray indices to render */
    const int64_t *sel;
} oracle_rays;

typedef struct {
    double *rgb;            /* [n_out][3] */
    double *T;              /* [n_out] or NULL */
    uint32_t *visit_log;    /* [n_out][visit_cap] or NULL */
    uint32_t visit_cap;
    uint32_t *visit_count;  /* [n_out] or NULL */
    double *visit_delta;    /* [n_out][visit_cap] or NULL */
    double *visit_weight;   /* [n_out][visit_cap] or NULL: T_j alpha_j */
    uint8_t *flags;         /* [n_out] or NULL: near-tie bits */
} oracle_out;

typedef struct {
    double t_in, t_out;
    int32_t leaf;
} seg;

typedef struct {
    seg *s;
    size_t n, cap;
    int near_face;
    int oom;
} segbuf;

static void seg_push(segbuf *b, double t0, double t1, int32_t leaf)
{
    if (b->n == b->cap) {
        size_t nc = b->cap ? 2 * b->cap : 256;
        seg *ns = (seg *)realloc(b->s, nc * sizeof(seg));
        if (!ns) { b->oom = 1; return; }
        b->s = ns;
        b->cap = nc;
    }
    b->s[b->n].t_in = t0;
    b->s[b->n].t_out = t1;
    b->s[b->n].leaf = leaf;
    b->n++;
}

/* Slab test of the ray against box [lo, hi], t clipped to [0, inf).
 * Returns t_out - t_in (may be negative or -inf). */
static double slab(const double o[3], const double d[3], const double lo[3], const double hi[3],
                   double *t_in, double *t_out, int *near_face)
{
    double a = 0.0, b = INFINITY;
    int miss = 0;
    for (int k = 0; k < 3; ++k) {
        if (d[k] != 0.0) {
            double t1 = (lo[k] - o[k]) / d[k], t2 = (hi[k] - o[k]) / d[k];
            double tn = t1 < t2 ? t1 : t2, tf = t1 < t2 ? t2 : t1;
            if (tn > a) a = tn;
            if (tf < b) b = tf;
        } else {
            if (fabs(o[k] - lo[k]) <= NEAR_FACE_EPS || fabs(o[k] - hi[k]) <= NEAR_FACE_EPS)
                *near_face = 1;
            if (o[k] < lo[k] || o[k] > hi[k]) miss = 1;
        }
    }
    *t_in = a;
    *t_out = b;
    return miss ? -INFINITY : b - a;
}

typedef struct {
    const otree *tr;
    const double *o, *d;
    double cell0; /* world size of the root cube */
    const double *amin;
} walk_ctx;

static void collect(const walk_ctx *w, int32_t node, int depth, uint32_t x, uint32_t y, uint32_t z,
                    segbuf *buf)
{
    double s = w->cell0 / (double)(1u << depth);
    double lo[3] = {w->amin[0] + x * s, w->amin[1] + y * s, w->amin[2] + z * s};
    double hi[3] = {lo[0] + s, lo[1] + s, lo[2] + s};
    double t0, t1;
    int nf = 0;
    double len = slab(w->o, w->d, lo, hi, &t0, &t1, &nf);
    const onode *n = &w->tr->nodes[node];
    if (n->leaf >= 0) {
        if (nf) buf->near_face = 1;
        if (len > -NEAR_FACE_EPS && len <= NEAR_FACE_EPS) buf->near_face = 1;
        if (len > 0.0) seg_push(buf, t0, t1, n->leaf);
        return;
    }
    if (!(len > -NEAR_FACE_EPS) && !nf) return;
    for (int oct = 0; oct < 8; ++oct) {
        int32_t c = n->child[oct];
        if (c < 0) continue;
        collect(w, c, depth + 1, 2 * x + ((oct >> 2) & 1), 2 * y + ((oct >> 1) & 1),
                2 * z + (oct & 1), buf);
    }
}

static int seg_cmp(const void *pa, const void *pb)
{
    const seg *a = (const seg *)pa, *b = (const seg *)pb;
    if (a->t_in < b->t_in) return -1;
    if (a->t_in > b->t_in) return 1;
    if (a->t_out < b->t_out) return -1;
    if (a->t_out > b->t_out) return 1;
    return (a->leaf > b->leaf) - (a->leaf < b->leaf);
}

static void camera_ray(const oracle_rays *r, int64_t idx, double o[3], double d[3])
{
    int64_t px = idx % r->width, py = idx / r->width;
    double f[3], rt[3], u[3];
    for (int k = 0; k < 3; ++k) f[k] = r->target[k] - r->eye[k];
    double fl = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (int k = 0; k < 3; ++k) f[k] /= fl;
    /* right = f x up, true up = right x f */
    rt[0] = f[1] * r->up[2] - f[2] * r->up[1];
    rt[1] = f[2] * r->up[0] - f[0] * r->up[2];
    rt[2] = f[0] * r->up[1] - f[1] * r->up[0];
    double rl = sqrt(rt[0] * rt[0] + rt[1] * rt[1] + rt[2] * rt[2]);
    for (int k = 0; k < 3; ++k) rt[k] /= rl;
    u[0] = rt[1] * f[2] - rt[2] * f[1];
    u[1] = rt[2] * f[0] - rt[0] * f[2];
    u[2] = rt[0] * f[1] - rt[1] * f[0];
    double th = tan(0.5 * r->fov_y_deg * M_PI / 180.0);
    double aspect = (double)r->width / (double)r->height;
    double sx = (2.0 * ((double)px + 0.5) / (double)r->width - 1.0) * th * aspect;
    double sy = (1.0 - 2.0 * ((double)py + 0.5) / (double)r->height) * th;
    for (int k = 0; k < 3; ++k) {
        o[k] = r->eye[k];
        d[k] = f[k] + sx * rt[k] + sy * u[k];
    }
}

typedef struct {
    const otree *tr;
    const oracle_scene *sc;
    const oracle_rays *rays;
    const oracle_out *out;
    int64_t n_out;
    int tid, nth;
    int status;
} job;

static void render_one(job *jb, int64_t j, segbuf *buf)
{
    const oracle_scene *sc = jb->sc;
    const oracle_rays *r = jb->rays;
    const oracle_out *out = jb->out;
    int64_t idx = r->sel ? r->sel[j] : j;
    double o[3], d[3], t_frame = r->t;
    if (r->mode == 0) {
        camera_ray(r, idx, o, d);
    } else {
        for (int k = 0; k < 3; ++k) { o[k] = r->o[3 * idx + k]; d[k] = r->d[3 * idx + k]; }
        if (r->t_per_ray) t_frame = r->t_per_ray[idx];
    }
    double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int k = 0; k < 3; ++k) d[k] /= dl;

    buf->n = 0;
    buf->near_face = 0;
    if (jb->tr->n_leaves > 0) {
        walk_ctx w = {jb->tr, o, d, sc->aabb_size, sc->aabb_min};
        collect(&w, 0, 0, 0, 0, 0, buf);
    }
    if (buf->oom) { jb->status = ORC_ERR_OOM; return; }
    qsort(buf->s, buf->n, sizeof(seg), seg_cmp);

    const int n1 = sc->n1, n2 = sc->n2, nsh = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    const int ncoef = n1 + 3 * nsh * n2;
    double b[64], Y[9];
    oracle_basis(n1 > n2 ? n1 : n2, t_frame, sc->period_T, b);
    oracle_sh(sc->sh_degree, d, Y);

    double C[3] = {0.0, 0.0, 0.0}, T = 1.0;
    int near_stop = 0;
    uint32_t nv = 0;
    double log_stop = sc->stop_T > 0.0 ? log(sc->stop_T) : 0.0;
    for (size_t s = 0; s < buf->n; ++s) {
        const float *k = sc->coeffs + (size_t)buf->s[s].leaf * ncoef;
        double delta = buf->s[s].t_out - buf->s[s].t_in;
        double sraw = 0.0;
        for (int i = 0; i < n1; ++i) sraw += (double)k[i] * b[i];
        double sigma = sraw > 0.0 ? sraw : 0.0;
        double col[3];
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int q = 0; q < nsh; ++q) {
                double zq = 0.0;
                for (int i = 0; i < n2; ++i) zq += (double)k[n1 + (c * nsh + q) * n2 + i] * b[i];
                acc += zq * Y[q];
            }
            col[c] = 1.0 / (1.0 + exp(-acc));
        }
        double alpha = 1.0 - exp(-sigma * delta);
        double wgt = T * alpha;
        for (int c = 0; c < 3; ++c) C[c] += wgt * col[c];
        if (nv < out->visit_cap) {
            size_t at = (size_t)j * out->visit_cap + nv;
            if (out->visit_log) out->visit_log[at] = (uint32_t)buf->s[s].leaf;
            if (out->visit_delta) out->visit_delta[at] = delta;
            if (out->visit_weight) out->visit_weight[at] = wgt;
        }
        nv++;
        T *= 1.0 - alpha;
        if (sc->stop_T > 0.0 && T > 0.0 && fabs(log(T) - log_stop) < NEAR_STOP_LOG_EPS) near_stop = 1;
        if (T < sc->stop_T) break;
    }
    for (int c = 0; c < 3; ++c) out->rgb[3 * j + c] = C[c] + T * sc->bg[c];
    if (out->T) out->T[j] = T;
    if (out->visit_count) out->visit_count[j] = nv;
    if (out->flags) out->flags[j] = (uint8_t)((buf->near_face ? 1 : 0) | (near_stop ? 2 : 0));
}

static void *worker(void *p)
{
    job *jb = (job *)p;
    segbuf buf = {0};
    const int64_t chunk = 16;
    for (int64_t s = (int64_t)jb->tid * chunk; s < jb->n_out; s += (int64_t)jb->nth * chunk) {
        int64_t e = s + chunk < jb->n_out ? s + chunk : jb->n_out;
        for (int64_t j = s; j < e && jb->status == ORC_OK; ++j) render_one(jb, j, &buf);
    }
    free(buf.s);
    return NULL;
}

/* Renders every selected ray; outputs are indexed by position in the
 * selection (or by ray index when no selection is given). */
int oracle_render(const void *tree, const oracle_scene *sc, const oracle_rays *rays,
                  const oracle_out *out, int n_threads)
{
    const otree *tr = (const otree *)tree;
    if (!tr || !sc || !rays || !out || !out->rgb) return ORC_ERR_ARG;
    if (sc->n1 < 1 || sc->n1 > 64 || sc->n2 < 1 || sc->n2 > 64 || sc->sh_degree < 0 ||
        sc->sh_degree > 2 || sc->period_T <= 0.0 || sc->aabb_size <= 0.0)
        return ORC_ERR_ARG;
    if (tr->n_leaves > 0 && !sc->coeffs) return ORC_ERR_ARG;
    int64_t n_all;
    if (rays->mode == 0) {
        if (rays->width < 0 || rays->height < 0) return ORC_ERR_ARG;
        n_all = (int64_t)rays->width * rays->height;
    } else if (rays->mode == 1) {
        if (rays->n < 0 || (rays->n > 0 && (!rays->o || !rays->d))) return ORC_ERR_ARG;
        n_all = rays->n;
    } else {
        return ORC_ERR_ARG;
    }
    int64_t n_out = rays->sel ? rays->n_sel : n_all;
    if (rays->sel)
        for (int64_t j = 0; j < n_out; ++j)
            if (rays->sel[j] < 0 || rays->sel[j] >= n_all) return ORC_ERR_ARG;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    job jobs[256];
    pthread_t th[256];
    for (int i = 0; i < n_threads; ++i) {
        jobs[i] = (job){tr, sc, rays, out, n_out, i, n_threads, ORC_OK};
    }
    if (n_threads == 1) {
        worker(&jobs[0]);
        return jobs[0].status;
    }
    int started = 0;
    for (int i = 0; i < n_threads; ++i) {
        if (pthread_create(&th[i], NULL, worker, &jobs[i]) != 0) break;
        started++;
    }
    for (int i = started; i < n_threads; ++i) worker(&jobs[i]);
    int st = ORC_OK;
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    for (int i = 0; i < n_threads; ++i)
        if (jobs[i].status != ORC_OK) st = jobs[i].status;
    return st;
}

/* ------------------------------------------------------------------------ */
/* Gradient of the render (Sec. 4.3: fine-tuning by back-propagation through
 * the IDFT, Eq. 13).  For loss L with dL/dC given per ray and channel, this
 * accumulates dL/dk into grad [n_leaves][ncoef] (canonical order, upload
 * ids).  The visited segment list (including the early stop) is held fixed,
 * i.e. it is treated as part of the function.  Per ray, with w_j = T_j a_j:
 *   dC/dc_j = w_j,  dC/dsigma_j = delta_j (T_{j+1} c_j - S_j),
 *   S_j = sum_{k>j} w_k c_k + T_end bg   (accumulated back to front),
 *   dc/du = c (1 - c), du/dz_{c,k} = Y_k, dz/dk_{c,k,i} = IDFT_i(t),
 *   dsigma/dk_sigma_i = IDFT_i(t) where sigma_raw > 0, else 0.
 * Single-threaded and O(segments) memory per ray: small cases only. */
int oracle_render_grad(const void *tree, const oracle_scene *sc, const oracle_rays *rays,
                       const double *dL_drgb, double *grad)
{
    const otree *tr = (const otree *)tree;
    if (!tr || !sc || !rays || !dL_drgb || !grad) return ORC_ERR_ARG;
    if (sc->n1 < 1 || sc->n1 > 64 || sc->n2 < 1 || sc->n2 > 64 || sc->sh_degree < 0 ||
        sc->sh_degree > 2 || sc->period_T <= 0.0 || sc->aabb_size <= 0.0)
        return ORC_ERR_ARG;
    int64_t n_all = rays->mode == 0 ? (int64_t)rays->width * rays->height : rays->n;
    int64_t n_out = rays->sel ? rays->n_sel : n_all;
    const int n1 = sc->n1, n2 = sc->n2, nsh = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    const int ncoef = n1 + 3 * nsh * n2;
    segbuf buf = {0};
    size_t cap = 0;
    double *col = NULL, *wgt = NULL, *Tb = NULL, *sraw = NULL, *del = NULL;
    int status = ORC_OK;
    for (int64_t j = 0; j < n_out && status == ORC_OK; ++j) {
        int64_t idx = rays->sel ? rays->sel[j] : j;
        double o[3], d[3], t_frame = rays->t;
        if (rays->mode == 0) {
            camera_ray(rays, idx, o, d);
        } else {
            for (int k = 0; k < 3; ++k) { o[k] = rays->o[3 * idx + k]; d[k] = rays->d[3 * idx + k]; }
            if (rays->t_per_ray) t_frame = rays->t_per_ray[idx];
        }
        double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int k = 0; k < 3; ++k) d[k] /= dl;
        buf.n = 0;
        buf.near_face = 0;
        if (tr->n_leaves > 0) {
            walk_ctx w = {tr, o, d, sc->aabb_size, sc->aabb_min};
            collect(&w, 0, 0, 0, 0, 0, &buf);
        }
        if (buf.oom) { status = ORC_ERR_OOM; break; }
        qsort(buf.s, buf.n, sizeof(seg), seg_cmp);
        if (buf.n + 1 > cap) {
            cap = buf.n + 1;
            col = (double *)realloc(col, 3 * cap * sizeof(double));
            wgt = (double *)realloc(wgt, cap * sizeof(double));
            Tb = (double *)realloc(Tb, (cap + 1) * sizeof(double));
            sraw = (double *)realloc(sraw, cap * sizeof(double));
            del = (double *)realloc(del, cap * sizeof(double));
            if (!col || !wgt || !Tb || !sraw || !del) { status = ORC_ERR_OOM; break; }
        }
        double b[64], Y[9];
        oracle_basis(n1 > n2 ? n1 : n2, t_frame, sc->period_T, b);
        oracle_sh(sc->sh_degree, d, Y);
        /* forward, keeping every segment's values */
        double T = 1.0;
        size_t used = 0;
        for (size_t s = 0; s < buf.n; ++s) {
            const float *k = sc->coeffs + (size_t)buf.s[s].leaf * ncoef;
            double delta = buf.s[s].t_out - buf.s[s].t_in, sr = 0.0;
            for (int i = 0; i < n1; ++i) sr += (double)k[i] * b[i];
            double sigma = sr > 0.0 ? sr : 0.0;
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int q = 0; q < nsh; ++q) {
                    double zq = 0.0;
                    for (int i = 0; i < n2; ++i) zq += (double)k[n1 + (c * nsh + q) * n2 + i] * b[i];
                    acc += zq * Y[q];
                }
                col[3 * s + c] = 1.0 / (1.0 + exp(-acc));
            }
            double alpha = 1.0 - exp(-sigma * delta);
            Tb[s] = T;
            wgt[s] = T * alpha;
            sraw[s] = sr;
            del[s] = delta;
            T *= 1.0 - alpha;
            used = s + 1;
            if (T < sc->stop_T) break;
        }
        Tb[used] = T;
        /* backward: S_j accumulated from the back */
        const double *g = dL_drgb + 3 * j;
        double S[3] = {T * sc->bg[0], T * sc->bg[1], T * sc->bg[2]};
        for (size_t s = used; s-- > 0;) {
            double *gk = grad + (size_t)buf.s[s].leaf * ncoef;
            double dsig = 0.0;
            for (int c = 0; c < 3; ++c) dsig += g[c] * del[s] * (Tb[s + 1] * col[3 * s + c] - S[c]);
            if (sraw[s] > 0.0)
                for (int i = 0; i < n1; ++i) gk[i] += dsig * b[i];
            for (int c = 0; c < 3; ++c) {
                double cc = col[3 * s + c];
                double du = g[c] * wgt[s] * cc * (1.0 - cc);
                for (int q = 0; q < nsh; ++q)
                    for (int i = 0; i < n2; ++i) gk[n1 + (c * nsh + q) * n2 + i] += du * Y[q] * b[i];
            }
            for (int c = 0; c < 3; ++c) S[c] += wgt[s] * col[3 * s + c];
        }
    }
    free(buf.s);
    free(col);
    free(wgt);
    free(Tb);
    free(sraw);
    free(del);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Eq. 10-12 (Sec. 4.2): per-leaf DFT of values sampled at frames t = 1..T,
 *   k_i = sum_{t=1}^{T} x(t) DFT_i(t),
 *   DFT_i(t) = (w_i / T) cos(i pi t / T) for even i, (w_i / T) sin((i+1) pi t / T) for odd i.
 * The paper prints w_i = 1; with it the inverse DFT of Eq. 7-9 would halve
 * every non-constant term, so this build reads w_0 = 1, w_i = 2 (i >= 1),
 * which makes Eq. 8 the exact inverse for signals of frequency < T/2.
 * x: [T][n_series]; k: [n_series][n_coef]. */
int oracle_dft(int T, int n_series, const double *x, int n_coef, double *k)
{
    if (T < 1 || n_series < 0 || n_coef < 1 || (n_series > 0 && (!x || !k))) return ORC_ERR_ARG;
    for (int s = 0; s < n_series; ++s) {
        for (int i = 0; i < n_coef; ++i) {
            double acc = 0.0;
            for (int t = 1; t <= T; ++t) {
                double basis = (i % 2 == 0) ? cos((double)i * M_PI * t / T)
                                            : sin((double)(i + 1) * M_PI * t / T);
                double w = i == 0 ? 1.0 : 2.0;
                acc += x[(size_t)(t - 1) * n_series + s] * (w / T) * basis;
            }
            k[(size_t)s * n_coef + i] = acc;
        }
    }
    return ORC_OK;
}
