/*
 * fv_oracle.c -- plain, slow, sequential FP64 CPU oracle of one PISO time step
 * and one SIMPLE iteration on a face-addressed finite-volume mesh.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; it is loaded by the tests, by the package's smoke check
 * and by the benchmark's CPU-baseline leg.  It shares no code, header, table
 * or helper with the CUDA path.
 *
 * What it follows (the paper, "Complete PISO and SIMPLE solvers on GPUs"):
 *   Sec. 3    PISO = momentum solve, then a series of pressure solves with
 *             explicit velocity corrections; SIMPLE = the same steps tuned for
 *             steady flow; FVM discretisation of the incompressible N-S
 *             equations; Jacobi-preconditioned CG for the pressure system and
 *             Jacobi-preconditioned BiCGStab for the non-symmetric momentum
 *             systems.
 *   Sec. 3.1  mesh model: N cells, each face shared by two cells or on the
 *             boundary; A_ij != 0 iff cells i and j share a face or i == j.
 *   Sec. 4.2  double precision throughout.
 * The paper gives no discretisation formulas; where it is silent the oracle
 * takes the textbook collocated finite-volume PISO/SIMPLE (the formulation the
 * paper says it follows), and every such choice is marked READING below.
 *
 * Arithmetic rules: straight sequential loops, sums in face order or cell
 * order, no blocking, no reordering.  Built with -O2 -ffp-contract=off.
 *
 * Parallel build (-fopenmp -DORC_PARALLEL, liborc_omp.so), used for the
 * full-size workloads and the timed CPU baseline: the same source with two
 * differences, both confined to the helpers marked ORC_PARALLEL below.
 *  (1) Dot products and norms sum fixed blocks of 4096 consecutive terms in
 *      element order and then add the block sums pairwise in block order, so
 *      the result does not depend on the number of threads; only the
 *      rounding of the sums differs from the sequential build.
 *  (2) Inside the Krylov solvers the LDU product runs row by row over
 *      threads, each row adding its terms in exactly the order of the
 *      sequential face loop (diagonal, then the faces where the row is the
 *      neighbour in face order, then the faces it owns in face order -- the
 *      order the face loop produces when internal faces are sorted by
 *      (owner, neighbour), as every oracle mesh's are); products are
 *      therefore bit-identical.  Element-wise vector updates run over
 *      threads with unchanged arithmetic.
 * Everything else (assembly, corrections, renumbering) stays sequential.
 *
 * Storage: vectors of 3 components are stored component-major (SoA):
 * x[c*n + i].  All arrays inside an omesh / ocase are in the renumbered
 * ("internal") cell and face order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { P_WALL = 0, P_INLET = 1, P_OUTLET = 2, P_EMPTY = 3 };

typedef struct {
    int type, start, size;
} opatch;

typedef struct {
    int N, F, B, np;
    int *own;           /* [F+B] */
    int *nei;           /* [F]   */
    double *Sf, *Cf;    /* [3*(F+B)] */
    double *C, *V;      /* [3*N], [N] */
    double *magSf;      /* [F+B] */
    double *w;          /* [F] owner interpolation weight */
    double *delta;      /* [F+B] */
    double *kv;         /* [3*F] non-orthogonal correction vector */
    int nonorth;
    opatch *patch;      /* [np] */
    int *bpatch;        /* [B] patch of each boundary face */
    int *cell_new_of_old, *face_new_of_old;
    signed char *flipped;
} omesh;

struct oamg_s;

typedef struct {
    omesh *m;
    double nu;
    double *u, *p, *phi;    /* [3N], [N], [F+B] */
    double *ub, *pb;        /* boundary-face values [3B], [B] */
    int psolver;            /* pressure solver: 0 Jacobi-CG, 1 multigrid-CG */
    struct oamg_s *amg;     /* multigrid hierarchy (built when selected) */
} ocase;

struct oamg_s *orc_amg_new(const omesh *m);
void orc_amg_free(struct oamg_s *h);
int orc_amg_pcg(struct oamg_s *h, const double *diag, const double *upper, const double *b,
                double *x, double tol, double reltol, int maxit, double *res0_out,
                double *res_out, int *iters_out);

/* ------------------------------------------------------------------------ */
/* small vector helpers (sequential)                                         */
/* ------------------------------------------------------------------------ */

#ifdef ORC_PARALLEL
#include <omp.h>
#define ORC_FOR _Pragma("omp parallel for schedule(static)")
enum { ORC_DOT_BLOCK = 4096 };

/* fixed-block dot product: block sums in element order, then pairwise
 * combination in block order (independent of the thread count) */
static double dot_n(int n, const double *a, const double *b)
{
    int nb = (n + ORC_DOT_BLOCK - 1) / ORC_DOT_BLOCK;
    if (nb <= 1) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += a[i] * b[i];
        return s;
    }
    double *part = malloc(sizeof(double) * (size_t)nb);
    if (!part) abort();
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nb; ++k) {
        int lo = k * ORC_DOT_BLOCK, hi = lo + ORC_DOT_BLOCK < n ? lo + ORC_DOT_BLOCK : n;
        double s = 0.0;
        for (int i = lo; i < hi; ++i) s += a[i] * b[i];
        part[k] = s;
    }
    while (nb > 1) {
        int h = nb / 2;
        for (int k = 0; k < h; ++k) part[k] = part[2 * k] + part[2 * k + 1];
        if (nb & 1) part[h] = part[nb - 1];
        nb = h + (nb & 1);
    }
    double s = part[0];
    free(part);
    return s;
}

void orc_set_threads(int n) { if (n > 0) omp_set_num_threads(n); }
int orc_threads(void) { return omp_get_max_threads(); }
#else
#define ORC_FOR
static double dot_n(int n, const double *a, const double *b)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

void orc_set_threads(int n) { (void)n; }
int orc_threads(void) { return 1; }
#endif
int orc_parallel_build(void)
{
#ifdef ORC_PARALLEL
    return 1;
#else
    return 0;
#endif
}

static double norm2_n(int n, const double *a) { return sqrt(dot_n(n, a, a)); }

static void *xcalloc(size_t n, size_t sz)
{
    void *p = calloc(n ? n : 1, sz);
    if (!p) abort();
    return p;
}

/* ------------------------------------------------------------------------ */
/* Reverse Cuthill-McKee renumbering.                                         */
/* READING (the paper only asks for a GPU-friendly data layout, Sec. 3.1):   */
/*  - graph = cells joined by internal faces;                                */
/*  - start: unvisited cell of minimum degree, ties -> lowest current index; */
/*  - BFS; the unvisited neighbours of each dequeued cell are appended in    */
/*    ascending (degree, index) order;                                       */
/*  - further components restart the same way; the whole order is reversed; */
/*  - no pseudo-peripheral search.                                           */
/* ------------------------------------------------------------------------ */

static const int *g_deg_for_sort;
static int cmp_deg_idx(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    if (g_deg_for_sort[x] != g_deg_for_sort[y]) return g_deg_for_sort[x] < g_deg_for_sort[y] ? -1 : 1;
    return (x > y) - (x < y);
}

static void rcm_order(int N, int F, const int *own, const int *nei, int *new_of_old)
{
    int *deg = xcalloc(N, sizeof(int));
    for (int f = 0; f < F; ++f) { deg[own[f]]++; deg[nei[f]]++; }
    int *start = xcalloc(N + 1, sizeof(int));
    for (int i = 0; i < N; ++i) start[i + 1] = start[i] + deg[i];
    int *fill = xcalloc(N, sizeof(int));
    int *adj = xcalloc(start[N], sizeof(int));
    for (int f = 0; f < F; ++f) {
        adj[start[own[f]] + fill[own[f]]++] = nei[f];
        adj[start[nei[f]] + fill[nei[f]]++] = own[f];
    }
    g_deg_for_sort = deg;
    for (int i = 0; i < N; ++i) qsort(adj + start[i], deg[i], sizeof(int), cmp_deg_idx);

    char *visited = xcalloc(N, 1);
    int *order = xcalloc(N, sizeof(int));
    int head = 0, tail = 0;
    while (tail < N) {
        int s = -1;
        for (int i = 0; i < N; ++i)
            if (!visited[i] && (s < 0 || deg[i] < deg[s])) s = i;
        visited[s] = 1;
        order[tail++] = s;
        while (head < tail) {
            int v = order[head++];
            for (int k = start[v]; k < start[v + 1]; ++k) {
                int u = adj[k];
                if (!visited[u]) { visited[u] = 1; order[tail++] = u; }
            }
        }
    }
    for (int pos = 0; pos < N; ++pos) new_of_old[order[N - 1 - pos]] = pos;
    free(deg); free(start); free(fill); free(adj); free(visited); free(order);
}

/* face sort keys */
typedef struct { long long k1, k2, k3; int idx; } fkey;
static int cmp_fkey(const void *a, const void *b)
{
    const fkey *x = a, *y = b;
    if (x->k1 != y->k1) return x->k1 < y->k1 ? -1 : 1;
    if (x->k2 != y->k2) return x->k2 < y->k2 ? -1 : 1;
    if (x->k3 != y->k3) return x->k3 < y->k3 ? -1 : 1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Mesh construction: renumbering, face orientation/order, geometry.          */
/* ------------------------------------------------------------------------ */

omesh *orc_mesh_new(int N, int F, int B, const int *own_in, const int *nei_in,
                    const double *Sf_in, const double *Cf_in, const double *C_in,
                    const double *V_in, int np, const int *ptype, const int *pstart,
                    const int *psize, int renumber)
{
    omesh *m = xcalloc(1, sizeof(omesh));
    int M = F + B;
    m->N = N; m->F = F; m->B = B; m->np = np;
    m->cell_new_of_old = xcalloc(N, sizeof(int));
    m->face_new_of_old = xcalloc(M, sizeof(int));
    m->flipped = xcalloc(M, 1);
    if (renumber) rcm_order(N, F, own_in, nei_in, m->cell_new_of_old);
    else for (int i = 0; i < N; ++i) m->cell_new_of_old[i] = i;
    const int *no = m->cell_new_of_old;

    /* internal faces: orient owner < neighbour, sort by (owner, neighbour) */
    fkey *keys = xcalloc(M, sizeof(fkey));
    for (int f = 0; f < F; ++f) {
        int a = no[own_in[f]], b = no[nei_in[f]];
        keys[f].k1 = a < b ? a : b;
        keys[f].k2 = a < b ? b : a;
        keys[f].k3 = f;
        keys[f].idx = f;
        m->flipped[f] = a > b;
    }
    qsort(keys, F, sizeof(fkey), cmp_fkey);
    for (int pos = 0; pos < F; ++pos) m->face_new_of_old[keys[pos].idx] = pos;
    /* boundary faces: sort by (patch, new owner, original index) */
    m->patch = xcalloc(np, sizeof(opatch));
    for (int b = 0; b < B; ++b) {
        int pat = -1;
        for (int q = 0; q < np; ++q)
            if (b >= pstart[q] && b < pstart[q] + psize[q]) pat = q;
        keys[b].k1 = pat;
        keys[b].k2 = no[own_in[F + b]];
        keys[b].k3 = b;
        keys[b].idx = b;
    }
    qsort(keys, B, sizeof(fkey), cmp_fkey);
    for (int pos = 0; pos < B; ++pos) m->face_new_of_old[F + keys[pos].idx] = F + pos;
    free(keys);
    for (int q = 0; q < np; ++q) {
        m->patch[q].type = ptype[q];
        m->patch[q].start = pstart[q];   /* the sort keeps every patch in place */
        m->patch[q].size = psize[q];
    }
    m->bpatch = xcalloc(B, sizeof(int));
    for (int q = 0; q < np; ++q)
        for (int j = 0; j < psize[q]; ++j) m->bpatch[pstart[q] + j] = q;

    /* renumbered arrays */
    m->own = xcalloc(M, sizeof(int));
    m->nei = xcalloc(F, sizeof(int));
    m->Sf = xcalloc(3 * (size_t)M, sizeof(double));
    m->Cf = xcalloc(3 * (size_t)M, sizeof(double));
    m->C = xcalloc(3 * (size_t)N, sizeof(double));
    m->V = xcalloc(N, sizeof(double));
    for (int f = 0; f < M; ++f) {
        int fn = m->face_new_of_old[f];
        double sgn = m->flipped[f] ? -1.0 : 1.0;
        if (f < F) {
            int a = no[own_in[f]], b = no[nei_in[f]];
            m->own[fn] = a < b ? a : b;
            m->nei[fn] = a < b ? b : a;
        } else {
            m->own[fn] = no[own_in[f]];
        }
        for (int c = 0; c < 3; ++c) {
            m->Sf[c * M + fn] = sgn * Sf_in[c * M + f];
            m->Cf[c * M + fn] = Cf_in[c * M + f];
        }
    }
    for (int i = 0; i < N; ++i) {
        for (int c = 0; c < 3; ++c) m->C[c * N + no[i]] = C_in[c * N + i];
        m->V[no[i]] = V_in[i];
    }

    /* geometry.  READINGS (the paper defers the discretisation to the
     * textbook finite-volume method):
     *  n = S/|S|, d = C_N - C_P;
     *  w = n.(C_N - Cf) / (n.(C_N - Cf) + n.(Cf - C_P))   (face value
     *      x_f = w x_P + (1-w) x_N);
     *  delta = 1 / max(n.d, 0.05 |d|);  k = n - delta d  (over-relaxed split
     *      S = |S| delta d + |S| k);
     *  boundary: d = Cf - C_P, delta = 1/max(n.d, 0.05|d|), no k. */
    m->magSf = xcalloc(M, sizeof(double));
    m->w = xcalloc(F ? F : 1, sizeof(double));
    m->delta = xcalloc(M, sizeof(double));
    m->kv = xcalloc(3 * (size_t)(F ? F : 1), sizeof(double));
    m->nonorth = 0;
    for (int f = 0; f < M; ++f) {
        double S[3], n[3], d[3], cf[3], cp[3];
        for (int c = 0; c < 3; ++c) {
            S[c] = m->Sf[c * M + f];
            cf[c] = m->Cf[c * M + f];
            cp[c] = m->C[c * N + m->own[f]];
        }
        double mag = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
        m->magSf[f] = mag;
        for (int c = 0; c < 3; ++c) n[c] = S[c] / mag;
        if (f < F) {
            double cn[3];
            for (int c = 0; c < 3; ++c) cn[c] = m->C[c * N + m->nei[f]];
            double a1 = 0.0, a2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                a1 += n[c] * (cn[c] - cf[c]);
                a2 += n[c] * (cf[c] - cp[c]);
            }
            m->w[f] = a1 / (a1 + a2);
            for (int c = 0; c < 3; ++c) d[c] = cn[c] - cp[c];
        } else {
            for (int c = 0; c < 3; ++c) d[c] = cf[c] - cp[c];
        }
        double nd = n[0] * d[0] + n[1] * d[1] + n[2] * d[2];
        double dm = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double den = nd > 0.05 * dm ? nd : 0.05 * dm;
        m->delta[f] = 1.0 / den;
        if (f < F) {
            double kk = 0.0;
            for (int c = 0; c < 3; ++c) {
                double k = n[c] - m->delta[f] * d[c];
                m->kv[c * F + f] = k;
                kk += k * k;
            }
            /* READING: the explicit non-orthogonal terms are switched on for a
             * mesh iff some internal face has |k| > 1e-8 (|k| is
             * dimensionless); on orthogonal hexahedra |k| is rounding noise. */
            if (sqrt(kk) > 1e-8) m->nonorth = 1;
        }
    }
    return m;
}

void orc_mesh_free(omesh *m)
{
    if (!m) return;
    free(m->own); free(m->nei); free(m->Sf); free(m->Cf); free(m->C); free(m->V);
    free(m->magSf); free(m->w); free(m->delta); free(m->kv); free(m->patch);
    free(m->bpatch); free(m->cell_new_of_old); free(m->face_new_of_old); free(m->flipped);
    free(m);
}

void orc_mesh_orders(const omesh *m, int *cell_new_of_old, int *face_new_of_old, signed char *flipped)
{
    memcpy(cell_new_of_old, m->cell_new_of_old, sizeof(int) * m->N);
    memcpy(face_new_of_old, m->face_new_of_old, sizeof(int) * (m->F + m->B));
    memcpy(flipped, m->flipped, m->F + m->B);
}

void orc_mesh_addressing(const omesh *m, int *own, int *nei)
{
    memcpy(own, m->own, sizeof(int) * (m->F + m->B));
    memcpy(nei, m->nei, sizeof(int) * m->F);
}

void orc_mesh_geometry(const omesh *m, double *magSf, double *w, double *delta, double *kv,
                       double *Sf, double *V)
{
    int M = m->F + m->B;
    memcpy(magSf, m->magSf, sizeof(double) * M);
    memcpy(w, m->w, sizeof(double) * m->F);
    memcpy(delta, m->delta, sizeof(double) * M);
    memcpy(kv, m->kv, sizeof(double) * 3 * m->F);
    memcpy(Sf, m->Sf, sizeof(double) * 3 * M);
    memcpy(V, m->V, sizeof(double) * m->N);
}

int orc_mesh_nonorth(const omesh *m) { return m->nonorth; }

/* ------------------------------------------------------------------------ */
/* LDU matrix-vector product (the paper's SMVP, Sec. 4.3.2):                  */
/* row P: diag_P x_P + sum_{f: own=P} upper_f x_nei + sum_{f: nei=P} lower_f x_own */
/* ------------------------------------------------------------------------ */

static void ldu_matvec(int N, int F, const int *own, const int *nei, const double *diag,
                       const double *upper, const double *lower, const double *x, double *y)
{
    for (int i = 0; i < N; ++i) y[i] = diag[i] * x[i];
    for (int f = 0; f < F; ++f) {
        y[own[f]] += upper[f] * x[nei[f]];
        y[nei[f]] += lower[f] * x[own[f]];
    }
}

void orc_ldu_matvec(int N, int F, const int *own, const int *nei, const double *diag,
                    const double *upper, const double *lower, const double *x, double *y)
{
    ldu_matvec(N, F, own, nei, diag, upper, lower, x, y);
}

/* The Krylov solvers' product.  Sequential build: the face loop above.
 * Parallel build (when the internal faces are sorted by (owner, neighbour)):
 * row i adds diag_i x_i, then lower_f x_own[f] over the faces whose
 * neighbour is i in face order, then upper_f x_nei[f] over the faces it owns
 * in face order -- the face loop's own order of additions into y_i. */
typedef struct {
    int ok;                  /* 1 when the row form is in use */
    int *lo_ptr, *lo_face;   /* faces with neighbour i: lo_face[lo_ptr[i] ..] */
    int *up_ptr;             /* faces owned by i: up_ptr[i] .. up_ptr[i+1]-1 */
} orows;

static void rows_init(orows *R, int N, int F, const int *own, const int *nei)
{
    memset(R, 0, sizeof(*R));
#ifdef ORC_PARALLEL
    for (int f = 1; f < F; ++f)
        if (own[f] < own[f - 1] || (own[f] == own[f - 1] && nei[f] <= nei[f - 1])) return;
    for (int f = 0; f < F; ++f)
        if (!(own[f] < nei[f]) || own[f] < 0 || nei[f] >= N) return;
    R->lo_ptr = xcalloc((size_t)N + 1, sizeof(int));
    R->lo_face = xcalloc(F ? F : 1, sizeof(int));
    R->up_ptr = xcalloc((size_t)N + 1, sizeof(int));
    for (int f = 0; f < F; ++f) { R->lo_ptr[nei[f] + 1]++; R->up_ptr[own[f] + 1]++; }
    for (int i = 0; i < N; ++i) {
        R->lo_ptr[i + 1] += R->lo_ptr[i];
        R->up_ptr[i + 1] += R->up_ptr[i];
    }
    int *fill = xcalloc((size_t)N, sizeof(int));
    for (int f = 0; f < F; ++f) R->lo_face[R->lo_ptr[nei[f]] + fill[nei[f]]++] = f;
    free(fill);
    R->ok = 1;
#else
    (void)N; (void)F; (void)own; (void)nei;
#endif
}

static void rows_free(orows *R)
{
    free(R->lo_ptr); free(R->lo_face); free(R->up_ptr);
}

static void krylov_matvec(const orows *R, int N, int F, const int *own, const int *nei,
                          const double *diag, const double *upper, const double *lower,
                          const double *x, double *y)
{
    if (!R->ok) {
        ldu_matvec(N, F, own, nei, diag, upper, lower, x, y);
        return;
    }
    ORC_FOR
    for (int i = 0; i < N; ++i) {
        double s = diag[i] * x[i];
        for (int k = R->lo_ptr[i]; k < R->lo_ptr[i + 1]; ++k) {
            int f = R->lo_face[k];
            s += lower[f] * x[own[f]];
        }
        for (int f = R->up_ptr[i]; f < R->up_ptr[i + 1]; ++f) s += upper[f] * x[nei[f]];
        y[i] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Jacobi-preconditioned CG (paper Sec. 3 and Sec. 4.3.2: SMVP, daxpy, dot,  */
/* reduction and the diagonal preconditioner).                               */
/* READING: warm start from x; stop when ||r||_2 <= max(tol ||b||_2,          */
/* reltol ||r_0||_2), r the recursively updated residual, tested before the  */
/* first iteration and after every r update; ||b|| = 0 returns x = 0.        */
/* Returns the iteration count (number of SMVPs); -1 if not converged,       */
/* -2 on breakdown (non-positive or non-finite curvature).                   */
/* ------------------------------------------------------------------------ */

int orc_pcg(int N, int F, const int *own, const int *nei, const double *diag,
            const double *upper, const double *b, double *x, double tol, double reltol,
            int maxit, double *res0_out, double *res_out, int *iters_out)
{
    double *r = xcalloc(N, sizeof(double)), *z = xcalloc(N, sizeof(double));
    double *p = xcalloc(N, sizeof(double)), *q = xcalloc(N, sizeof(double));
    int status = 0, it = 0;
    double nb = norm2_n(N, b);
    if (nb == 0.0) {
        for (int i = 0; i < N; ++i) x[i] = 0.0;
        *res0_out = 0.0; *res_out = 0.0; *iters_out = 0;
        free(r); free(z); free(p); free(q);
        return 0;
    }
    orows R;
    rows_init(&R, N, F, own, nei);
    krylov_matvec(&R, N, F, own, nei, diag, upper, upper, x, q);
    ORC_FOR
    for (int i = 0; i < N; ++i) r[i] = b[i] - q[i];
    double nr = norm2_n(N, r);
    double thresh = tol * nb;
    if (reltol * nr > thresh) thresh = reltol * nr;
    *res0_out = nr / nb;
    if (nr <= thresh) goto done;
    ORC_FOR
    for (int i = 0; i < N; ++i) z[i] = r[i] / diag[i];
    ORC_FOR
    for (int i = 0; i < N; ++i) p[i] = z[i];
    double rho = dot_n(N, r, z);
    for (it = 1; it <= maxit; ++it) {
        krylov_matvec(&R, N, F, own, nei, diag, upper, upper, p, q);
        double pq = dot_n(N, p, q);
        if (!(pq > 0.0) || !isfinite(pq)) { status = -2; break; }
        double alpha = rho / pq;
        ORC_FOR
        for (int i = 0; i < N; ++i) x[i] += alpha * p[i];
        ORC_FOR
        for (int i = 0; i < N; ++i) r[i] -= alpha * q[i];
        nr = norm2_n(N, r);
        if (!isfinite(nr)) { status = -2; break; }
        if (nr <= thresh) break;
        if (it == maxit) { status = -1; break; }
        ORC_FOR
        for (int i = 0; i < N; ++i) z[i] = r[i] / diag[i];
        double rho_new = dot_n(N, r, z);
        double beta = rho_new / rho;
        rho = rho_new;
        ORC_FOR
        for (int i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
    }
    if (it > maxit) status = -1;
done:
    *res_out = nr / nb;
    *iters_out = it > maxit ? maxit : it;
    rows_free(&R);
    free(r); free(z); free(p); free(q);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Jacobi (right) preconditioned BiCGStab of van der Vorst for the momentum  */
/* systems (paper Sec. 3).  Shadow residual r^ = r_0.                         */
/* READING: same stopping rule as CG, tested before the first iteration and  */
/* after each full iteration (no half-step exit); ||b|| = 0 returns x = 0.    */
/* ------------------------------------------------------------------------ */

int orc_bicgstab(int N, int F, const int *own, const int *nei, const double *diag,
                 const double *upper, const double *lower, const double *b, double *x,
                 double tol, double reltol, int maxit, double *res0_out, double *res_out,
                 int *iters_out)
{
    double *r = xcalloc(N, sizeof(double)), *rh = xcalloc(N, sizeof(double));
    double *p = xcalloc(N, sizeof(double)), *v = xcalloc(N, sizeof(double));
    double *y = xcalloc(N, sizeof(double)), *s = xcalloc(N, sizeof(double));
    double *z = xcalloc(N, sizeof(double)), *t = xcalloc(N, sizeof(double));
    int status = 0, it = 0;
    double nb = norm2_n(N, b), nr = 0.0;
    if (nb == 0.0) {
        for (int i = 0; i < N; ++i) x[i] = 0.0;
        *res0_out = 0.0; *res_out = 0.0; *iters_out = 0;
        goto out;
    }
    orows R;
    rows_init(&R, N, F, own, nei);
    krylov_matvec(&R, N, F, own, nei, diag, upper, lower, x, t);
    ORC_FOR
    for (int i = 0; i < N; ++i) { r[i] = b[i] - t[i]; rh[i] = r[i]; }
    nr = norm2_n(N, r);
    double thresh = tol * nb;
    if (reltol * nr > thresh) thresh = reltol * nr;
    *res0_out = nr / nb;
    if (nr <= thresh) goto done;
    double rho_old = 1.0, alpha = 1.0, omega = 1.0;
    for (it = 1; it <= maxit; ++it) {
        double rho = dot_n(N, rh, r);
        if (it == 1) {
            ORC_FOR
            for (int i = 0; i < N; ++i) p[i] = r[i];
        } else {
            double beta = (rho / rho_old) * (alpha / omega);
            ORC_FOR
            for (int i = 0; i < N; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
        }
        ORC_FOR
        for (int i = 0; i < N; ++i) y[i] = p[i] / diag[i];
        krylov_matvec(&R, N, F, own, nei, diag, upper, lower, y, v);
        double rv = dot_n(N, rh, v);
        if (rv == 0.0 || !isfinite(rv)) { status = -2; break; }
        alpha = rho / rv;
        ORC_FOR
        for (int i = 0; i < N; ++i) s[i] = r[i] - alpha * v[i];
        ORC_FOR
        for (int i = 0; i < N; ++i) z[i] = s[i] / diag[i];
        krylov_matvec(&R, N, F, own, nei, diag, upper, lower, z, t);
        double ts = dot_n(N, t, s), tt = dot_n(N, t, t);
        omega = tt > 0.0 ? ts / tt : 0.0;
        ORC_FOR
        for (int i = 0; i < N; ++i) x[i] += alpha * y[i] + omega * z[i];
        ORC_FOR
        for (int i = 0; i < N; ++i) r[i] = s[i] - omega * t[i];
        nr = norm2_n(N, r);
        if (!isfinite(nr)) { status = -2; break; }
        if (nr <= thresh) break;
        if (it == maxit) { status = -1; break; }
        if (omega == 0.0) { status = -2; break; }
        rho_old = rho;
    }
    if (it > maxit) status = -1;
done:
    *res_out = nr / nb;
    *iters_out = it > maxit ? maxit : it;
    rows_free(&R);
out:
    free(r); free(rh); free(p); free(v); free(y); free(s); free(z); free(t);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Dense Gaussian elimination with partial pivoting (pin for the Krylov      */
/* solvers on tiny meshes).  A is n x n row-major, overwritten; b := A^-1 b. */
/* ------------------------------------------------------------------------ */

int orc_dense_solve(int n, double *A, double *b)
{
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[(size_t)i * n + k]) > fabs(A[(size_t)piv * n + k])) piv = i;
        if (A[(size_t)piv * n + k] == 0.0) return -1;
        if (piv != k) {
            for (int j = 0; j < n; ++j) {
                double t = A[(size_t)k * n + j];
                A[(size_t)k * n + j] = A[(size_t)piv * n + j];
                A[(size_t)piv * n + j] = t;
            }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            double l = A[(size_t)i * n + k] / A[(size_t)k * n + k];
            for (int j = k; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
            b[i] -= l * b[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < n; ++j) s -= A[(size_t)k * n + j] * b[j];
        b[k] = s / A[(size_t)k * n + k];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Case (fields + boundary values)                                            */
/* ------------------------------------------------------------------------ */

ocase *orc_case_new(omesh *m, double nu)
{
    ocase *cs = xcalloc(1, sizeof(ocase));
    cs->m = m;
    cs->nu = nu;
    cs->u = xcalloc(3 * (size_t)m->N, sizeof(double));
    cs->p = xcalloc(m->N, sizeof(double));
    cs->phi = xcalloc(m->F + m->B, sizeof(double));
    cs->ub = xcalloc(3 * (size_t)(m->B ? m->B : 1), sizeof(double));
    cs->pb = xcalloc(m->B ? m->B : 1, sizeof(double));
    return cs;
}

void orc_case_free(ocase *cs)
{
    if (!cs) return;
    free(cs->u); free(cs->p); free(cs->phi); free(cs->ub); free(cs->pb);
    orc_amg_free(cs->amg);
    free(cs);
}

/* fields in the caller's (original) order when original_order != 0:
 * u [3][N], p [N], phi [F+B] with the caller's face orientation. */
void orc_case_set_fields(ocase *cs, const double *u, const double *p, const double *phi,
                         int original_order)
{
    const omesh *m = cs->m;
    int N = m->N, M = m->F + m->B;
    for (int i = 0; i < N; ++i) {
        int j = original_order ? m->cell_new_of_old[i] : i;
        for (int c = 0; c < 3; ++c) cs->u[c * N + j] = u[c * N + i];
        cs->p[j] = p[i];
    }
    for (int f = 0; f < M; ++f) {
        int g = original_order ? m->face_new_of_old[f] : f;
        double s = (original_order && m->flipped[f]) ? -1.0 : 1.0;
        cs->phi[g] = s * phi[f];
    }
}

void orc_case_get_fields(const ocase *cs, double *u, double *p, double *phi, int original_order)
{
    const omesh *m = cs->m;
    int N = m->N, M = m->F + m->B;
    for (int i = 0; i < N; ++i) {
        int j = original_order ? m->cell_new_of_old[i] : i;
        for (int c = 0; c < 3; ++c) u[c * N + i] = cs->u[c * N + j];
        p[i] = cs->p[j];
    }
    for (int f = 0; f < M; ++f) {
        int g = original_order ? m->face_new_of_old[f] : f;
        double s = (original_order && m->flipped[f]) ? -1.0 : 1.0;
        phi[f] = s * cs->phi[g];
    }
}

/* Uniform value on one patch (time-dependent boundary conditions, Sec. 1/6). */
void orc_patch_set_value(ocase *cs, int q, const double *u3, double p)
{
    const omesh *m = cs->m;
    for (int j = 0; j < m->patch[q].size; ++j) {
        int b = m->patch[q].start + j;
        for (int c = 0; c < 3; ++c) cs->ub[c * m->B + b] = u3[c];
        cs->pb[b] = p;
    }
}

/* Per-face values on one patch, given in the caller's face order within the
 * patch: u [3][size], p [size] (p may be NULL). */
void orc_patch_set_face_values(ocase *cs, int q, const double *u, const double *p)
{
    const omesh *m = cs->m;
    int size = m->patch[q].size;
    for (int j = 0; j < size; ++j) {
        int b = m->face_new_of_old[m->F + m->patch[q].start + j] - m->F;
        for (int c = 0; c < 3; ++c) cs->ub[c * m->B + b] = u[c * size + j];
        if (p) cs->pb[b] = p[j];
    }
}

/* ------------------------------------------------------------------------ */
/* Finite-volume operators (paper Sec. 4.3.3: gradient, divergence,           */
/* Laplacian).                                                                */
/* ------------------------------------------------------------------------ */

/* Gauss gradient: grad x_P = (1/V_P) [ sum_int (+-S_f) x_f + sum_bnd S_b x_b ],
 * x_f = w x_P + (1-w) x_N; empty faces are skipped. */
static void gauss_grad(const omesh *m, const double *x, const double *xb, double *g)
{
    int N = m->N, F = m->F, B = m->B, M = F + B;
    for (int i = 0; i < 3 * N; ++i) g[i] = 0.0;
    for (int f = 0; f < F; ++f) {
        int P = m->own[f], Q = m->nei[f];
        double xf = m->w[f] * x[P] + (1.0 - m->w[f]) * x[Q];
        for (int c = 0; c < 3; ++c) {
            g[c * N + P] += m->Sf[c * M + f] * xf;
            g[c * N + Q] -= m->Sf[c * M + f] * xf;
        }
    }
    for (int b = 0; b < B; ++b) {
        int fb = F + b;
        if (m->patch[m->bpatch[b]].type == P_EMPTY) continue;
        int P = m->own[fb];
        for (int c = 0; c < 3; ++c) g[c * N + P] += m->Sf[c * M + fb] * xb[b];
    }
    for (int c = 0; c < 3; ++c)
        for (int i = 0; i < N; ++i) g[c * N + i] /= m->V[i];
}

/* boundary values of p: fixed on outlets, zero-gradient elsewhere */
static void p_boundary(const ocase *cs, const double *p, double *xb)
{
    const omesh *m = cs->m;
    for (int b = 0; b < m->B; ++b) {
        int t = m->patch[m->bpatch[b]].type;
        xb[b] = (t == P_OUTLET) ? cs->pb[b] : p[m->own[m->F + b]];
    }
}

/* boundary values of velocity component c: fixed on walls and inlets,
 * zero-gradient on outlets */
static void u_boundary(const ocase *cs, int c, const double *uc, double *xb)
{
    const omesh *m = cs->m;
    for (int b = 0; b < m->B; ++b) {
        int t = m->patch[m->bpatch[b]].type;
        xb[b] = (t == P_WALL || t == P_INLET) ? cs->ub[c * m->B + b] : uc[m->own[m->F + b]];
    }
}

static void grad_p(const ocase *cs, const double *p, double *g)
{
    double *xb = xcalloc(cs->m->B, sizeof(double));
    p_boundary(cs, p, xb);
    gauss_grad(cs->m, p, xb, g);
    free(xb);
}

/* gradU [9N]: component-major, gradU[(3c + d) N + i] = d u_c / d x_d */
static void grad_u(const ocase *cs, double *gU)
{
    const omesh *m = cs->m;
    int N = m->N;
    double *xb = xcalloc(m->B, sizeof(double));
    for (int c = 0; c < 3; ++c) {
        u_boundary(cs, c, cs->u + (size_t)c * N, xb);
        gauss_grad(m, cs->u + (size_t)c * N, xb, gU + (size_t)3 * c * N);
    }
    free(xb);
}

void orc_case_grad_p(const ocase *cs, double *g) { grad_p(cs, cs->p, g); }

/* ------------------------------------------------------------------------ */
/* Momentum matrix M (LDU) and source (paper Sec. 3: the momentum equation   */
/* solved first in PISO/SIMPLE).  READINGS:                                   */
/*  ddt (PISO): Euler implicit, diag += V/dt, src += V/dt u^n;                */
/*  convection: central ("linear") face value, flux F = phi_f out of P:       */
/*     diag_P += F w, upper += F (1-w); diag_N -= F (1-w), lower -= F w;      */
/*  diffusion D = nu |S| delta: diag_P += D, diag_N += D, upper -= D,         */
/*     lower -= D; explicit non-orthogonal term nu |S| k.(grad u)_f added to  */
/*     src_P and subtracted from src_N (gradient of the current u);           */
/*  fixed-U boundary: src += (nu |S| delta_b - F_b) u_b, diag += nu|S|delta_b;*/
/*  outlet (zero-gradient U): diag += F_b;                                     */
/*  SIMPLE: no ddt; implicit relaxation diag' = diag/alpha,                   */
/*     src += (diag' - diag) u_prev.                                           */
/* The pressure gradient is NOT part of src.                                   */
/* ------------------------------------------------------------------------ */

static void assemble_momentum(const ocase *cs, int transient, double dt, double alpha_u,
                              const double *gU, double *diag, double *upper, double *lower,
                              double *src)
{
    const omesh *m = cs->m;
    int N = m->N, F = m->F, B = m->B, M = F + B;
    double nu = cs->nu;
    for (int i = 0; i < N; ++i) diag[i] = 0.0;
    for (int i = 0; i < 3 * N; ++i) src[i] = 0.0;
    for (int f = 0; f < F; ++f) { upper[f] = 0.0; lower[f] = 0.0; }
    if (transient) {
        for (int i = 0; i < N; ++i) {
            double vdt = m->V[i] / dt;
            diag[i] += vdt;
            for (int c = 0; c < 3; ++c) src[c * N + i] += vdt * cs->u[c * N + i];
        }
    }
    for (int f = 0; f < F; ++f) {
        int P = m->own[f], Q = m->nei[f];
        double Fl = cs->phi[f], w = m->w[f];
        diag[P] += Fl * w;
        upper[f] += Fl * (1.0 - w);
        diag[Q] -= Fl * (1.0 - w);
        lower[f] -= Fl * w;
        double D = nu * m->magSf[f] * m->delta[f];
        diag[P] += D;
        diag[Q] += D;
        upper[f] -= D;
        lower[f] -= D;
        if (m->nonorth) {
            for (int c = 0; c < 3; ++c) {
                double kg = 0.0;
                for (int d = 0; d < 3; ++d) {
                    double gf = w * gU[(3 * c + d) * N + P] + (1.0 - w) * gU[(3 * c + d) * N + Q];
                    kg += m->kv[d * F + f] * gf;
                }
                double t = nu * m->magSf[f] * kg;
                src[c * N + P] += t;
                src[c * N + Q] -= t;
            }
        }
    }
    for (int b = 0; b < B; ++b) {
        int fb = F + b, P = m->own[fb];
        int t = m->patch[m->bpatch[b]].type;
        if (t == P_EMPTY) continue;
        if (t == P_WALL || t == P_INLET) {
            double D = nu * m->magSf[fb] * m->delta[fb];
            double Fb = cs->phi[fb];
            diag[P] += D;
            for (int c = 0; c < 3; ++c) {
                double ubc = cs->ub[c * B + b];
                src[c * N + P] += D * ubc - Fb * ubc;
            }
        } else if (t == P_OUTLET) {
            diag[P] += cs->phi[fb];
        }
    }
    (void)M;
    if (!transient) {
        for (int i = 0; i < N; ++i) {
            double d0 = diag[i], d1 = d0 / alpha_u;
            diag[i] = d1;
            for (int c = 0; c < 3; ++c) src[c * N + i] += (d1 - d0) * cs->u[c * N + i];
        }
    }
}

void orc_case_momentum_system(const ocase *cs, int transient, double dt, double alpha_u,
                              double *diag, double *upper, double *lower, double *src)
{
    const omesh *m = cs->m;
    double *gU = m->nonorth ? xcalloc(9 * (size_t)m->N, sizeof(double)) : NULL;
    if (gU) grad_u(cs, gU);
    assemble_momentum(cs, transient, dt, alpha_u, gU, diag, upper, lower, src);
    free(gU);
}

/* ------------------------------------------------------------------------ */
/* Pressure step pieces (paper Sec. 3: pressure solve + explicit velocity    */
/* correction).  READINGS:                                                    */
/*  A_P = diag of M; H_P = src_P - sum offdiag u_nbr; HbyA = H/A;             */
/*  rAU = V/A; phi*_f = (interp HbyA)_f . S_f (no time-derivative flux term); */
/*  boundary phi*: fixed-U -> u_b.S_b, outlet -> HbyA_P.S_b;                  */
/*  pressure matrix = negated Laplacian of rAU (SPD): a_f = rAU_f |S| delta,  */
/*  rAU_f = w rAU_P + (1-w) rAU_N, diag += a_f both sides, upper = -a_f;      */
/*  fixed-p (outlet) face: a_b = rAU_P |S| delta_b, diag += a_b, b += a_b p_b;*/
/*  b_P = -sum_out phi*  + sum_out rAU_f |S| k.(grad p)_f (lagged gradient);  */
/*  reference cell r (closed domains): b_r += diag_r p_ref, diag_r *= 2;      */
/*  flux: phi_f = phi*_f - a_f (p_N - p_P) - rAU_f |S| k.(grad p)_f,          */
/*        outlet phi_b = phi*_b - a_b (p_b - p_P);                            */
/*  velocity: u = HbyA - rAU grad p.                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    double *HbyA, *rAU, *phis, *af, *nof, *pdiag, *pup, *pb;
} pwork;

static void pwork_alloc(pwork *w, const omesh *m)
{
    int N = m->N, M = m->F + m->B;
    w->HbyA = xcalloc(3 * (size_t)N, sizeof(double));
    w->rAU = xcalloc(N, sizeof(double));
    w->phis = xcalloc(M, sizeof(double));
    w->af = xcalloc(M, sizeof(double));
    w->nof = xcalloc(m->F ? m->F : 1, sizeof(double));
    w->pdiag = xcalloc(N, sizeof(double));
    w->pup = xcalloc(m->F ? m->F : 1, sizeof(double));
    w->pb = xcalloc(N, sizeof(double));
}

static void pwork_free(pwork *w)
{
    free(w->HbyA); free(w->rAU); free(w->phis); free(w->af); free(w->nof);
    free(w->pdiag); free(w->pup); free(w->pb);
}

static void compute_HbyA(const ocase *cs, const double *mdiag, const double *upper,
                         const double *lower, const double *src, pwork *w)
{
    const omesh *m = cs->m;
    int N = m->N, F = m->F;
    for (int c = 0; c < 3; ++c) {
        double *H = w->HbyA + (size_t)c * N;
        const double *uc = cs->u + (size_t)c * N;
        for (int i = 0; i < N; ++i) H[i] = src[c * N + i];
        for (int f = 0; f < F; ++f) {
            H[m->own[f]] -= upper[f] * uc[m->nei[f]];
            H[m->nei[f]] -= lower[f] * uc[m->own[f]];
        }
        for (int i = 0; i < N; ++i) H[i] /= mdiag[i];
    }
    for (int i = 0; i < N; ++i) w->rAU[i] = m->V[i] / mdiag[i];
}

static void assemble_pressure(const ocase *cs, const double *gradp, int ref_cell, double p_ref,
                              pwork *w)
{
    const omesh *m = cs->m;
    int N = m->N, F = m->F, B = m->B, M = F + B;
    for (int i = 0; i < N; ++i) { w->pdiag[i] = 0.0; w->pb[i] = 0.0; }
    for (int f = 0; f < M; ++f) { w->phis[f] = 0.0; w->af[f] = 0.0; }
    for (int f = 0; f < F; ++f) {
        int P = m->own[f], Q = m->nei[f];
        double wf = m->w[f];
        double ph = 0.0;
        for (int c = 0; c < 3; ++c) {
            double hf = wf * w->HbyA[c * N + P] + (1.0 - wf) * w->HbyA[c * N + Q];
            ph += hf * m->Sf[c * M + f];
        }
        w->phis[f] = ph;
        double rf = wf * w->rAU[P] + (1.0 - wf) * w->rAU[Q];
        double a = rf * m->magSf[f] * m->delta[f];
        w->af[f] = a;
        w->pdiag[P] += a;
        w->pdiag[Q] += a;
        w->pup[f] = -a;
        w->pb[P] -= ph;
        w->pb[Q] += ph;
        w->nof[f] = 0.0;
        if (m->nonorth) {
            double kg = 0.0;
            for (int d = 0; d < 3; ++d) {
                double gf = wf * gradp[d * N + P] + (1.0 - wf) * gradp[d * N + Q];
                kg += m->kv[d * F + f] * gf;
            }
            double nf = rf * m->magSf[f] * kg;
            w->nof[f] = nf;
            w->pb[P] += nf;
            w->pb[Q] -= nf;
        }
    }
    for (int b = 0; b < B; ++b) {
        int fb = F + b, P = m->own[fb];
        int t = m->patch[m->bpatch[b]].type;
        if (t == P_EMPTY) continue;
        double ph = 0.0;
        if (t == P_WALL || t == P_INLET) {
            for (int c = 0; c < 3; ++c) ph += cs->ub[c * B + b] * m->Sf[c * M + fb];
        } else {
            for (int c = 0; c < 3; ++c) ph += w->HbyA[c * N + P] * m->Sf[c * M + fb];
            double a = w->rAU[P] * m->magSf[fb] * m->delta[fb];
            w->af[fb] = a;
            w->pdiag[P] += a;
            w->pb[P] += a * cs->pb[b];
        }
        w->phis[fb] = ph;
        w->pb[P] -= ph;
    }
    if (ref_cell >= 0) {
        w->pb[ref_cell] += w->pdiag[ref_cell] * p_ref;
        w->pdiag[ref_cell] *= 2.0;
    }
}

static void correct_flux(ocase *cs, const pwork *w)
{
    const omesh *m = cs->m;
    int F = m->F, B = m->B;
    const double *p = cs->p;
    for (int f = 0; f < F; ++f)
        cs->phi[f] = w->phis[f] - w->af[f] * (p[m->nei[f]] - p[m->own[f]]) - w->nof[f];
    for (int b = 0; b < B; ++b) {
        int fb = F + b;
        int t = m->patch[m->bpatch[b]].type;
        if (t == P_EMPTY) cs->phi[fb] = 0.0;
        else if (t == P_OUTLET) cs->phi[fb] = w->phis[fb] - w->af[fb] * (cs->pb[b] - p[m->own[fb]]);
        else cs->phi[fb] = w->phis[fb];
    }
}

/* max_P | sum_out phi_P + (b - A p)_P + pin_P | / max|b|; identity of the
 * flux correction (pin_P = diag_r/2 (p_r - p_ref) at the reference cell). */
static double continuity_identity(const ocase *cs, const pwork *w, int ref_cell, double p_ref)
{
    const omesh *m = cs->m;
    int N = m->N, F = m->F, B = m->B;
    double *div = xcalloc(N, sizeof(double)), *Ap = xcalloc(N, sizeof(double));
    for (int f = 0; f < F; ++f) { div[m->own[f]] += cs->phi[f]; div[m->nei[f]] -= cs->phi[f]; }
    for (int b = 0; b < B; ++b) div[m->own[F + b]] += cs->phi[F + b];
    ldu_matvec(N, F, m->own, m->nei, w->pdiag, w->pup, w->pup, cs->p, Ap);
    double mb = 0.0, me = 0.0;
    for (int i = 0; i < N; ++i) if (fabs(w->pb[i]) > mb) mb = fabs(w->pb[i]);
    for (int i = 0; i < N; ++i) {
        double e = div[i] + (w->pb[i] - Ap[i]);
        if (i == ref_cell) e += 0.5 * w->pdiag[i] * (cs->p[i] - p_ref);
        if (fabs(e) > me) me = fabs(e);
    }
    free(div); free(Ap);
    return mb > 0.0 ? me / mb : me;
}

static void correct_velocity(ocase *cs, const pwork *w, double *gradp)
{
    const omesh *m = cs->m;
    int N = m->N;
    grad_p(cs, cs->p, gradp);
    for (int c = 0; c < 3; ++c)
        for (int i = 0; i < N; ++i)
            cs->u[c * N + i] = w->HbyA[c * N + i] - w->rAU[i] * gradp[c * N + i];
}

/* The pressure solve of a corrector: Jacobi-CG, or CG preconditioned by   */
/* the aggregation-multigrid V-cycle when the case selects it.               */
static int pressure_solve(ocase *cs, const pwork *w, double tol, double reltol, int maxit,
                          double *res0, double *res1, int *iters)
{
    const omesh *m = cs->m;
    if (cs->psolver == 1)
        return orc_amg_pcg(cs->amg, w->pdiag, w->pup, w->pb, cs->p, tol, reltol, maxit, res0,
                           res1, iters);
    return orc_pcg(m->N, m->F, m->own, m->nei, w->pdiag, w->pup, w->pb, cs->p, tol, reltol,
                   maxit, res0, res1, iters);
}

/* select the pressure solver: 0 Jacobi-CG, 1 multigrid-CG */
int orc_case_set_pressure_solver(ocase *cs, int solver)
{
    if (solver != 0 && solver != 1) return -1;
    if (solver == 1 && !cs->amg) cs->amg = orc_amg_new(cs->m);
    cs->psolver = solver;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* PISO time step (paper Sec. 3): momentum predictor, then n_corr pressure   */
/* corrections.  M is assembled once per step; H uses the current u.         */
/* Each corrector solves the pressure equation 1 + n_nonorth times: after a  */
/* solve, the explicit non-orthogonal part of the right-hand side (and of    */
/* the face flux) is re-evaluated with the gradient of the new pressure and  */
/* the equation solved again from that pressure (the non-orthogonal          */
/* correctors of the textbook method; the paper's Sec. 5 notes their cost on */
/* the non-orthogonal artery mesh).  The flux is corrected after the last.   */
/* Per-solve statistics: iters[0..2] momentum components, then one entry per */
/* pressure solve in order (corrector k, loop j at 3 + k (1 + n_nonorth) + j);*/
/* res[2k] initial and res[2k+1] final normalised residual of solve k.       */
/* Returns 0, or the first non-zero solver status.                            */
/* ------------------------------------------------------------------------ */

/* p_sched (may be NULL): for replaying another implementation's run, the
 * number of iterations each pressure solve takes, in the order of iters[3..]
 * (the solve then runs exactly that many CG iterations: tolerance 0, limit
 * p_sched[k]); the arithmetic of every iteration is unchanged. */
static int piso_step_impl(ocase *cs, double dt, int n_corr, int n_nonorth, double p_tol,
                          int p_maxit, double u_tol, int u_maxit, int ref_orig, double p_ref,
                          int *iters, double *res, double *cont_err, const int *p_sched)
{
    const omesh *m = cs->m;
    int N = m->N, F = m->F;
    int ref = ref_orig >= 0 ? m->cell_new_of_old[ref_orig] : -1;
    int status = 0, st;
    double *gradp = xcalloc(3 * (size_t)N, sizeof(double));
    double *gU = m->nonorth ? xcalloc(9 * (size_t)N, sizeof(double)) : NULL;
    double *mdiag = xcalloc(N, sizeof(double)), *up = xcalloc(F ? F : 1, sizeof(double));
    double *lo = xcalloc(F ? F : 1, sizeof(double)), *src = xcalloc(3 * (size_t)N, sizeof(double));
    double *rhs = xcalloc(N, sizeof(double));
    pwork w;
    pwork_alloc(&w, m);

    grad_p(cs, cs->p, gradp);
    if (gU) grad_u(cs, gU);
    assemble_momentum(cs, 1, dt, 1.0, gU, mdiag, up, lo, src);
    for (int c = 0; c < 3; ++c) {
        for (int i = 0; i < N; ++i) rhs[i] = src[c * N + i] - m->V[i] * gradp[c * N + i];
        st = orc_bicgstab(N, F, m->own, m->nei, mdiag, up, lo, rhs, cs->u + (size_t)c * N,
                          u_tol, 0.0, u_maxit, &res[2 * c], &res[2 * c + 1], &iters[c]);
        if (st && !status) status = st;
    }
    *cont_err = 0.0;
    for (int k = 0; k < n_corr; ++k) {
        compute_HbyA(cs, mdiag, up, lo, src, &w);
        for (int j = 0; j <= n_nonorth; ++j) {
            const int sk = 3 + k * (n_nonorth + 1) + j;
            if (j > 0) grad_p(cs, cs->p, gradp);
            assemble_pressure(cs, gradp, ref, p_ref, &w);
            if (p_sched)
                st = pressure_solve(cs, &w, 0.0, 0.0, p_sched[sk - 3], &res[2 * sk],
                                    &res[2 * sk + 1], &iters[sk]);
            else
                st = pressure_solve(cs, &w, p_tol, 0.0, p_maxit, &res[2 * sk], &res[2 * sk + 1],
                                    &iters[sk]);
            if (st && !status) status = st;
        }
        correct_flux(cs, &w);
        double ce = continuity_identity(cs, &w, ref, p_ref);
        if (ce > *cont_err) *cont_err = ce;
        correct_velocity(cs, &w, gradp);
    }
    pwork_free(&w);
    free(gradp); free(gU); free(mdiag); free(up); free(lo); free(src); free(rhs);
    return status;
}

int orc_piso_step(ocase *cs, double dt, int n_corr, int n_nonorth, double p_tol, int p_maxit,
                  double u_tol, int u_maxit, int ref_orig, double p_ref, int *iters, double *res,
                  double *cont_err)
{
    return piso_step_impl(cs, dt, n_corr, n_nonorth, p_tol, p_maxit, u_tol, u_maxit, ref_orig,
                          p_ref, iters, res, cont_err, NULL);
}

/* The PISO step with every pressure solve held to a given iteration count
 * (p_sched [n_corr (1 + n_nonorth)]); a solve whose count is reached reports
 * status -1 like any iteration-limited solve. */
int orc_piso_step_sched(ocase *cs, double dt, int n_corr, int n_nonorth, double u_tol,
                        int u_maxit, int ref_orig, double p_ref, const int *p_sched, int *iters,
                        double *res, double *cont_err)
{
    return piso_step_impl(cs, dt, n_corr, n_nonorth, 0.0, 0, u_tol, u_maxit, ref_orig, p_ref,
                          iters, res, cont_err, p_sched);
}

/* ------------------------------------------------------------------------ */
/* SIMPLE iteration (paper Sec. 3).  READINGS: implicit momentum relaxation  */
/* alpha_u; 1 + n_nonorth pressure solves (non-orthogonal correctors as in   */
/* the PISO step); the flux is corrected with the unrelaxed                  */
/* pressure; then p <- p_old + alpha_p (p_sol - p_old) and                    */
/* u = HbyA - rAU grad p_relaxed.  Outer convergence measure init_res_max =   */
/* max of                                                                      */
/*   max_c ||b_c - M u_c||_2 / max_c ||b_c||_2   (momentum, before the solve) */
/*   ||b_p - A p||_2 / ||phi*||_2                (pressure, before the solve) */
/* i.e. each equation's initial residual scaled by a quantity that does not   */
/* vanish when a component of the exact solution is zero.                     */
/* ------------------------------------------------------------------------ */

int orc_simple_iter(ocase *cs, double alpha_u, double alpha_p, int n_nonorth, double p_tol,
                    double p_reltol, int p_maxit, double u_tol, double u_reltol, int u_maxit,
                    int ref_orig, double p_ref, int *iters, double *res, double *cont_err,
                    double *init_res_max)
{
    const omesh *m = cs->m;
    int N = m->N, F = m->F;
    int ref = ref_orig >= 0 ? m->cell_new_of_old[ref_orig] : -1;
    int status = 0, st;
    double *gradp = xcalloc(3 * (size_t)N, sizeof(double));
    double *gU = m->nonorth ? xcalloc(9 * (size_t)N, sizeof(double)) : NULL;
    double *mdiag = xcalloc(N, sizeof(double)), *up = xcalloc(F ? F : 1, sizeof(double));
    double *lo = xcalloc(F ? F : 1, sizeof(double)), *src = xcalloc(3 * (size_t)N, sizeof(double));
    double *rhs = xcalloc(N, sizeof(double)), *pold = xcalloc(N, sizeof(double));
    pwork w;
    pwork_alloc(&w, m);
    double irm = 0.0;

    grad_p(cs, cs->p, gradp);
    if (gU) grad_u(cs, gU);
    assemble_momentum(cs, 0, 1.0, alpha_u, gU, mdiag, up, lo, src);
    double bmax = 0.0, rmax = 0.0;
    for (int c = 0; c < 3; ++c) {
        for (int i = 0; i < N; ++i) rhs[i] = src[c * N + i] - m->V[i] * gradp[c * N + i];
        ldu_matvec(N, F, m->own, m->nei, mdiag, up, lo, cs->u + (size_t)c * N, pold);
        for (int i = 0; i < N; ++i) pold[i] = rhs[i] - pold[i];
        double nb = norm2_n(N, rhs), nr = norm2_n(N, pold);
        if (nb > bmax) bmax = nb;
        if (nr > rmax) rmax = nr;
        st = orc_bicgstab(N, F, m->own, m->nei, mdiag, up, lo, rhs, cs->u + (size_t)c * N,
                          u_tol, u_reltol, u_maxit, &res[2 * c], &res[2 * c + 1], &iters[c]);
        if (st && !status) status = st;
    }
    if (bmax > 0.0) irm = rmax / bmax;
    compute_HbyA(cs, mdiag, up, lo, src, &w);
    assemble_pressure(cs, gradp, ref, p_ref, &w);
    {
        ldu_matvec(N, F, m->own, m->nei, w.pdiag, w.pup, w.pup, cs->p, pold);
        for (int i = 0; i < N; ++i) pold[i] = w.pb[i] - pold[i];
        double nr = norm2_n(N, pold), nphi = norm2_n(F + m->B, w.phis);
        double rp = nphi > 0.0 ? nr / nphi : nr;
        if (rp > irm) irm = rp;
    }
    memcpy(pold, cs->p, sizeof(double) * N);
    for (int j = 0; j <= n_nonorth; ++j) {
        if (j > 0) {
            grad_p(cs, cs->p, gradp);
            assemble_pressure(cs, gradp, ref, p_ref, &w);
        }
        st = pressure_solve(cs, &w, p_tol, p_reltol, p_maxit, &res[2 * (3 + j)],
                            &res[2 * (3 + j) + 1], &iters[3 + j]);
        if (st && !status) status = st;
    }
    correct_flux(cs, &w);
    *cont_err = continuity_identity(cs, &w, ref, p_ref);
    for (int i = 0; i < N; ++i) cs->p[i] = pold[i] + alpha_p * (cs->p[i] - pold[i]);
    correct_velocity(cs, &w, gradp);
    *init_res_max = irm;
    pwork_free(&w);
    free(gradp); free(gU); free(mdiag); free(up); free(lo); free(src); free(rhs); free(pold);
    return status;
}

/* Pressure system of the first PISO corrector from the current state (used
 * by the Krylov pins): returns diag [N], upper [F], b [N] in internal order. */
void orc_case_pressure_system(ocase *cs, double dt, int ref_orig, double p_ref, double *pdiag,
                              double *pup, double *pb)
{
    const omesh *m = cs->m;
    int N = m->N, F = m->F;
    int ref = ref_orig >= 0 ? m->cell_new_of_old[ref_orig] : -1;
    double *gradp = xcalloc(3 * (size_t)N, sizeof(double));
    double *gU = m->nonorth ? xcalloc(9 * (size_t)N, sizeof(double)) : NULL;
    double *mdiag = xcalloc(N, sizeof(double)), *up = xcalloc(F ? F : 1, sizeof(double));
    double *lo = xcalloc(F ? F : 1, sizeof(double)), *src = xcalloc(3 * (size_t)N, sizeof(double));
    pwork w;
    pwork_alloc(&w, m);
    grad_p(cs, cs->p, gradp);
    if (gU) grad_u(cs, gU);
    assemble_momentum(cs, 1, dt, 1.0, gU, mdiag, up, lo, src);
    compute_HbyA(cs, mdiag, up, lo, src, &w);
    assemble_pressure(cs, gradp, ref, p_ref, &w);
    memcpy(pdiag, w.pdiag, sizeof(double) * N);
    memcpy(pup, w.pup, sizeof(double) * F);
    memcpy(pb, w.pb, sizeof(double) * N);
    pwork_free(&w);
    free(gradp); free(gU); free(mdiag); free(up); free(lo); free(src);
}

/* Scalar Laplacian with Dirichlet boundary values (manufactured-solution
 * pin of the face-gradient discretisation, Sec. 4.3.3 "Laplacian"):
 * assembles  -div(grad x) V-integrated with x_b given on every non-empty
 * boundary face, non-orthogonal correction with the gradient of xg (lagged),
 * as diag [N], upper [F], b [N]. */
void orc_laplacian_system(const omesh *m, const double *xb, const double *gradx, double *diag,
                          double *upper, double *b)
{
    int N = m->N, F = m->F, B = m->B;
    for (int i = 0; i < N; ++i) { diag[i] = 0.0; b[i] = 0.0; }
    for (int f = 0; f < F; ++f) {
        int P = m->own[f], Q = m->nei[f];
        double a = m->magSf[f] * m->delta[f];
        diag[P] += a; diag[Q] += a; upper[f] = -a;
        if (m->nonorth && gradx) {
            double kg = 0.0;
            for (int d = 0; d < 3; ++d) {
                double gf = m->w[f] * gradx[d * N + P] + (1.0 - m->w[f]) * gradx[d * N + Q];
                kg += m->kv[d * F + f] * gf;
            }
            double nf = m->magSf[f] * kg;
            b[P] += nf; b[Q] -= nf;
        }
    }
    for (int q = 0; q < B; ++q) {
        int fb = F + q, P = m->own[fb];
        if (m->patch[m->bpatch[q]].type == P_EMPTY) continue;
        double a = m->magSf[fb] * m->delta[fb];
        diag[P] += a;
        b[P] += a * xb[q];
    }
}

/* Gauss gradient of a cell field with given boundary values (internal order). */
void orc_gauss_grad(const omesh *m, const double *x, const double *xb, double *g)
{
    gauss_grad(m, x, xb, g);
}

/* internal-order state access for tests */
void orc_case_state(const ocase *cs, double *u, double *p, double *phi)
{
    const omesh *m = cs->m;
    memcpy(u, cs->u, sizeof(double) * 3 * m->N);
    memcpy(p, cs->p, sizeof(double) * m->N);
    memcpy(phi, cs->phi, sizeof(double) * (m->F + m->B));
}

/* ------------------------------------------------------------------------ */
/* Hybrid ELL + J (+ CRS overflow) storage of a structurally symmetric       */
/* sparsity pattern (paper Sec. 3.1).  Input rows: row_ptr[n+1], col[]       */
/* ascending within a row, diagonal included.  Row-major N x K arrays as in  */
/* the paper's example:                                                      */
/*   ELL: the first K entries of row i; I[i K + k] = column, -1 = empty slot; */
/*   J[i K + k] = k' with I[j K + k'] = i, j = I[i K + k] (the slot of the    */
/*   transposed entry in row j); when that entry is in the CRS part at       */
/*   position p, J = -2 - p; empty slot: J = -1.                               */
/*   CRS: the entries of a row after its K-th, crs_ptr[n+1], crs_col[], and   */
/*   crs_tr[p] = the transposed entry's ELL slot (>= 0) or -2 - p'.           */
/* With crs_col == NULL only crs_ptr is filled.  Returns the number of CRS    */
/* entries, or -1 if some entry has no transpose (pattern not symmetric).     */
/* ------------------------------------------------------------------------ */

static int ellj_locate(const int *row_ptr, const int *col, int K, const int *crs_ptr, int j,
                       int i)
{
    /* position of entry (j, i): ELL slot k (>= 0) or -2 - p in the CRS part */
    int len = row_ptr[j + 1] - row_ptr[j];
    for (int t = 0; t < len; ++t) {
        if (col[row_ptr[j] + t] != i) continue;
        if (t < K) return t;
        return -2 - (crs_ptr[j] + (t - K));
    }
    return -1;
}

int orc_ellj_build(int n, const int *row_ptr, const int *col, int K, int *I, int *J,
                   int *crs_ptr, int *crs_col, int *crs_tr)
{
    crs_ptr[0] = 0;
    for (int i = 0; i < n; ++i) {
        int len = row_ptr[i + 1] - row_ptr[i];
        crs_ptr[i + 1] = crs_ptr[i] + (len > K ? len - K : 0);
    }
    int ncrs = crs_ptr[n];
    if (crs_col == NULL) return ncrs;
    for (int i = 0; i < n; ++i) {
        int len = row_ptr[i + 1] - row_ptr[i];
        for (int k = 0; k < K; ++k) {
            if (k < len) {
                int j = col[row_ptr[i] + k];
                int loc = ellj_locate(row_ptr, col, K, crs_ptr, j, i);
                if (loc == -1) return -1;
                I[(size_t)i * K + k] = j;
                J[(size_t)i * K + k] = loc;
            } else {
                I[(size_t)i * K + k] = -1;
                J[(size_t)i * K + k] = -1;
            }
        }
        for (int t = K; t < len; ++t) {
            int j = col[row_ptr[i] + t];
            int p = crs_ptr[i] + (t - K);
            int loc = ellj_locate(row_ptr, col, K, crs_ptr, j, i);
            if (loc == -1) return -1;
            crs_col[p] = j;
            crs_tr[p] = loc;
        }
    }
    return ncrs;
}

/* ------------------------------------------------------------------------ */
/* Aggregation multigrid preconditioner for the pressure CG (the stronger     */
/* pressure solver the paper's Sec. 5 and 6 call for; the paper itself runs  */
/* only Jacobi-CG on the GPU and compares with OpenFOAM's GAMG on the CPU).   */
/*                                                                            */
/* Setup, from the mesh alone: level 0 is the cell graph with edge weights    */
/* |S_f| Delta_f (the face coefficient of the Laplacian without rAU).  A      */
/* level's aggregates come from two pairwise-matching passes; each pass      */
/* visits the nodes in index order and pairs an unassigned node with its     */
/* unassigned neighbour of largest weight, or, when all its neighbours are   */
/* taken, adds it to the aggregate of its strongest neighbour (a node with   */
/* no neighbour stays alone).  Weights within a relative 1e-9 count as equal */
/* and the lower index wins.  The coarse graph joins two aggregates that     */
/* share a fine edge, with the summed weight; its edges are ordered by       */
/* (lower, higher) aggregate.  Coarsening stops at <= 32 nodes or when a     */
/* level shrinks by less than 10 %; the last level is solved directly.        */
/*                                                                            */
/* Per matrix (symmetric LDU: diag, upper): Galerkin coarse matrices with     */
/* piecewise-constant prolongation, A_c = P^T A P: a coarse diagonal sums the */
/* members' diagonals (ascending) and twice the coefficients of the faces    */
/* inside the aggregate (ascending); a coarse face sums its fine faces'       */
/* coefficients (ascending).  The coarsest matrix is factored by Cholesky.   */
/*                                                                            */
/* V-cycle z = M r: per level, from x = 0, nu = 2 weighted-Jacobi sweeps      */
/* x += omega (b - A x) / diag (omega = 2/3), the residual restricted by     */
/* summing over each aggregate, the coarse problem solved by the same cycle, */
/* the correction added with the over-correction factor alpha = 1.8 (the     */
/* plain piecewise-constant correction is too small in energy; alpha < 2     */
/* keeps the cycle symmetric positive definite), and nu = 2 sweeps again.    */
/* ------------------------------------------------------------------------ */

#define AMG_MAXLEV 24
#define AMG_OMEGA (2.0 / 3.0)
#define AMG_ALPHA 1.8
#define AMG_NU 2
#define AMG_NMIN 32
#define AMG_TIE 1e-9

typedef struct oamg_s {
    int nlev;
    int n[AMG_MAXLEV], ne[AMG_MAXLEV];
    int *ea[AMG_MAXLEV], *eb[AMG_MAXLEV];    /* edges of level l, ea < eb */
    int *agg[AMG_MAXLEV];                    /* level l node -> level l+1 node */
    int *emap[AMG_MAXLEV];                   /* level l edge -> level l+1 edge or -1 */
    double *d[AMG_MAXLEV], *o[AMG_MAXLEV];   /* current matrices */
    double *chol;                            /* coarsest Cholesky factor, row-major */
} oamg;

static int amg_better(double wc, int jc, double wb, int jb)
{
    if (jb < 0) return 1;
    if (wc > wb * (1.0 + AMG_TIE)) return 1;
    if (wc >= wb * (1.0 - AMG_TIE) && jc < jb) return 1;
    return 0;
}

/* one pairwise-matching pass over a graph; returns the number of aggregates */
static int amg_pass(int n, int ne, const int *ea, const int *eb, const double *ew, int *assign)
{
    int *deg = xcalloc(n + 1, sizeof(int));
    for (int e = 0; e < ne; ++e) { deg[ea[e] + 1]++; deg[eb[e] + 1]++; }
    for (int i = 0; i < n; ++i) deg[i + 1] += deg[i];
    int *fill = xcalloc(n, sizeof(int)), *adj = xcalloc(2 * (size_t)ne + 1, sizeof(int));
    double *aw = xcalloc(2 * (size_t)ne + 1, sizeof(double));
    for (int e = 0; e < ne; ++e) {
        int a = ea[e], b = eb[e];
        adj[deg[a] + fill[a]] = b; aw[deg[a] + fill[a]++] = ew[e];
        adj[deg[b] + fill[b]] = a; aw[deg[b] + fill[b]++] = ew[e];
    }
    for (int i = 0; i < n; ++i) assign[i] = -1;
    int na = 0;
    for (int i = 0; i < n; ++i) {
        if (assign[i] >= 0) continue;
        int bj = -1; double bw = 0.0;
        for (int t = deg[i]; t < deg[i + 1]; ++t)
            if (assign[adj[t]] < 0 && amg_better(aw[t], adj[t], bw, bj)) { bj = adj[t]; bw = aw[t]; }
        if (bj >= 0) { assign[i] = assign[bj] = na++; continue; }
        bj = -1; bw = 0.0;
        for (int t = deg[i]; t < deg[i + 1]; ++t)
            if (amg_better(aw[t], adj[t], bw, bj)) { bj = adj[t]; bw = aw[t]; }
        assign[i] = bj >= 0 ? assign[bj] : na++;
    }
    free(deg); free(fill); free(adj); free(aw);
    return na;
}

typedef struct { int lo, hi, e; } amg_key;

static int amg_key_cmp(const void *x, const void *y)
{
    const amg_key *a = x, *b = y;
    if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;
    if (a->hi != b->hi) return a->hi < b->hi ? -1 : 1;
    return a->e < b->e ? -1 : (a->e > b->e);
}

/* coarse graph of an assignment: edges, summed weights, fine edge -> coarse */
static int amg_coarse_graph(int ne, const int *ea, const int *eb, const double *ew,
                            const int *assign, int **cea, int **ceb, double **cew, int *emap)
{
    amg_key *k = xcalloc(ne + 1, sizeof(amg_key));
    int m = 0;
    for (int e = 0; e < ne; ++e) {
        int a = assign[ea[e]], b = assign[eb[e]];
        if (a == b) { emap[e] = -1; continue; }
        k[m].lo = a < b ? a : b; k[m].hi = a < b ? b : a; k[m].e = e; ++m;
    }
    qsort(k, m, sizeof(amg_key), amg_key_cmp);
    int nc = 0;
    for (int t = 0; t < m; ++t)
        if (t == 0 || k[t].lo != k[t - 1].lo || k[t].hi != k[t - 1].hi) ++nc;
    *cea = xcalloc(nc + 1, sizeof(int)); *ceb = xcalloc(nc + 1, sizeof(int));
    *cew = xcalloc(nc + 1, sizeof(double));
    int c = -1;
    for (int t = 0; t < m; ++t) {
        if (t == 0 || k[t].lo != k[t - 1].lo || k[t].hi != k[t - 1].hi) {
            ++c; (*cea)[c] = k[t].lo; (*ceb)[c] = k[t].hi; (*cew)[c] = 0.0;
        }
        emap[k[t].e] = c;
    }
    /* weights summed in ascending fine-edge order */
    for (int e = 0; e < ne; ++e) if (emap[e] >= 0) (*cew)[emap[e]] += ew[e];
    free(k);
    return nc;
}

oamg *orc_amg_new(const omesh *m)
{
    oamg *h = xcalloc(1, sizeof(oamg));
    int n = m->N, ne = m->F;
    int *ea = xcalloc(ne + 1, sizeof(int)), *eb = xcalloc(ne + 1, sizeof(int));
    double *ew = xcalloc(ne + 1, sizeof(double));
    for (int f = 0; f < ne; ++f) {
        ea[f] = m->own[f]; eb[f] = m->nei[f];
        ew[f] = m->magSf[f] * m->delta[f];
    }
    int l = 0;
    for (;;) {
        h->n[l] = n; h->ne[l] = ne; h->ea[l] = ea; h->eb[l] = eb;
        h->d[l] = xcalloc(n + 1, sizeof(double)); h->o[l] = xcalloc(ne + 1, sizeof(double));
        if (n <= AMG_NMIN || l + 1 >= AMG_MAXLEV) { free(ew); break; }
        int *a1 = xcalloc(n + 1, sizeof(int)), *m1 = xcalloc(ne + 1, sizeof(int));
        int n1 = amg_pass(n, ne, ea, eb, ew, a1);
        int *ea1, *eb1; double *ew1;
        int ne1 = amg_coarse_graph(ne, ea, eb, ew, a1, &ea1, &eb1, &ew1, m1);
        int *a2 = xcalloc(n1 + 1, sizeof(int)), *m2 = xcalloc(ne1 + 1, sizeof(int));
        int n2 = amg_pass(n1, ne1, ea1, eb1, ew1, a2);
        int *ea2, *eb2; double *ew2;
        int ne2 = amg_coarse_graph(ne1, ea1, eb1, ew1, a2, &ea2, &eb2, &ew2, m2);
        free(ea1); free(eb1); free(ew1);
        if ((double)n2 > 0.9 * n) {
            free(a1); free(m1); free(a2); free(m2); free(ea2); free(eb2); free(ew2); free(ew);
            break;
        }
        h->agg[l] = xcalloc(n + 1, sizeof(int));
        h->emap[l] = xcalloc(ne + 1, sizeof(int));
        for (int i = 0; i < n; ++i) h->agg[l][i] = a2[a1[i]];
        for (int e = 0; e < ne; ++e) h->emap[l][e] = m1[e] < 0 ? -1 : m2[m1[e]];
        free(a1); free(m1); free(a2); free(m2); free(ew);
        n = n2; ne = ne2; ea = ea2; eb = eb2; ew = ew2;
        ++l;
    }
    h->nlev = l + 1;
    int nc = h->n[l];
    h->chol = xcalloc((size_t)nc * nc + 1, sizeof(double));
    return h;
}

void orc_amg_free(oamg *h)
{
    if (!h) return;
    for (int l = 0; l < h->nlev; ++l) {
        free(h->ea[l]); free(h->eb[l]); free(h->agg[l]); free(h->emap[l]);
        free(h->d[l]); free(h->o[l]);
    }
    free(h->chol);
    free(h);
}

int orc_amg_levels(const oamg *h, int *n, int *ne)
{
    for (int l = 0; l < h->nlev; ++l) { n[l] = h->n[l]; ne[l] = h->ne[l]; }
    return h->nlev;
}

/* aggregate map and edge map of level l (l < nlev - 1) */
void orc_amg_maps(const oamg *h, int l, int *agg, int *emap)
{
    memcpy(agg, h->agg[l], sizeof(int) * h->n[l]);
    memcpy(emap, h->emap[l], sizeof(int) * h->ne[l]);
}

/* Galerkin coarse matrices and the coarsest factor; returns -1 if the
 * coarsest matrix is not positive definite. */
static int amg_set_matrix(oamg *h, const double *diag, const double *upper)
{
    memcpy(h->d[0], diag, sizeof(double) * h->n[0]);
    memcpy(h->o[0], upper, sizeof(double) * h->ne[0]);
    for (int l = 0; l + 1 < h->nlev; ++l) {
        double *cd = h->d[l + 1], *co = h->o[l + 1];
        for (int I = 0; I < h->n[l + 1]; ++I) cd[I] = 0.0;
        for (int E = 0; E < h->ne[l + 1]; ++E) co[E] = 0.0;
        for (int i = 0; i < h->n[l]; ++i) cd[h->agg[l][i]] += h->d[l][i];
        for (int e = 0; e < h->ne[l]; ++e)
            if (h->emap[l][e] < 0) cd[h->agg[l][h->ea[l][e]]] += 2.0 * h->o[l][e];
        for (int e = 0; e < h->ne[l]; ++e)
            if (h->emap[l][e] >= 0) co[h->emap[l][e]] += h->o[l][e];
    }
    int L = h->nlev - 1, n = h->n[L];
    double *c = h->chol;
    for (size_t t = 0; t < (size_t)n * n; ++t) c[t] = 0.0;
    for (int i = 0; i < n; ++i) c[(size_t)i * n + i] = h->d[L][i];
    for (int e = 0; e < h->ne[L]; ++e) {
        c[(size_t)h->ea[L][e] * n + h->eb[L][e]] = h->o[L][e];
        c[(size_t)h->eb[L][e] * n + h->ea[L][e]] = h->o[L][e];
    }
    /* Cholesky A = L L^T, L stored in the lower triangle */
    for (int j = 0; j < n; ++j) {
        double s = c[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= c[(size_t)j * n + k] * c[(size_t)j * n + k];
        if (!(s > 0.0)) return -1;
        double ljj = sqrt(s);
        c[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double t = c[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= c[(size_t)i * n + k] * c[(size_t)j * n + k];
            c[(size_t)i * n + j] = t / ljj;
        }
    }
    return 0;
}

static void amg_sweep(const oamg *h, int l, const double *b, double *x, double *t)
{
    int n = h->n[l];
    ldu_matvec(n, h->ne[l], h->ea[l], h->eb[l], h->d[l], h->o[l], h->o[l], x, t);
    for (int i = 0; i < n; ++i) x[i] += AMG_OMEGA * (b[i] - t[i]) / h->d[l][i];
}

static void amg_vcycle(const oamg *h, int l, const double *b, double *x)
{
    int n = h->n[l];
    if (l == h->nlev - 1) {
        const double *c = h->chol;
        for (int i = 0; i < n; ++i) {            /* L y = b */
            double s = b[i];
            for (int k = 0; k < i; ++k) s -= c[(size_t)i * n + k] * x[k];
            x[i] = s / c[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {       /* L^T x = y */
            double s = x[i];
            for (int k = i + 1; k < n; ++k) s -= c[(size_t)k * n + i] * x[k];
            x[i] = s / c[(size_t)i * n + i];
        }
        return;
    }
    double *t = xcalloc(n + 1, sizeof(double));
    for (int i = 0; i < n; ++i) x[i] = AMG_OMEGA * b[i] / h->d[l][i];
    for (int s = 1; s < AMG_NU; ++s) amg_sweep(h, l, b, x, t);
    ldu_matvec(n, h->ne[l], h->ea[l], h->eb[l], h->d[l], h->o[l], h->o[l], x, t);
    int nc = h->n[l + 1];
    double *bc = xcalloc(nc + 1, sizeof(double)), *xc = xcalloc(nc + 1, sizeof(double));
    for (int i = 0; i < n; ++i) bc[h->agg[l][i]] += b[i] - t[i];
    amg_vcycle(h, l + 1, bc, xc);
    for (int i = 0; i < n; ++i) x[i] += AMG_ALPHA * xc[h->agg[l][i]];
    for (int s = 0; s < AMG_NU; ++s) amg_sweep(h, l, b, x, t);
    free(t); free(bc); free(xc);
}

/* one V-cycle z = M r for the matrix (diag, upper); returns -1 if the
 * coarsest matrix is not positive definite */
int orc_amg_vcycle(oamg *h, const double *diag, const double *upper, const double *r, double *z)
{
    if (amg_set_matrix(h, diag, upper)) return -1;
    amg_vcycle(h, 0, r, z);
    return 0;
}

/* CG preconditioned by the V-cycle; the stopping rule, warm start and
 * statistics are those of orc_pcg. */
int orc_amg_pcg(oamg *h, const double *diag, const double *upper, const double *b, double *x,
                double tol, double reltol, int maxit, double *res0_out, double *res_out,
                int *iters_out)
{
    int N = h->n[0], F = h->ne[0];
    const int *own = h->ea[0], *nei = h->eb[0];
    double *r = xcalloc(N, sizeof(double)), *z = xcalloc(N, sizeof(double));
    double *p = xcalloc(N, sizeof(double)), *q = xcalloc(N, sizeof(double));
    int status = 0, it = 0;
    double nb = norm2_n(N, b);
    if (nb == 0.0) {
        for (int i = 0; i < N; ++i) x[i] = 0.0;
        *res0_out = 0.0; *res_out = 0.0; *iters_out = 0;
        free(r); free(z); free(p); free(q);
        return 0;
    }
    if (amg_set_matrix(h, diag, upper)) {
        *res0_out = *res_out = 0.0; *iters_out = 0;
        free(r); free(z); free(p); free(q);
        return -2;
    }
    ldu_matvec(N, F, own, nei, diag, upper, upper, x, q);
    for (int i = 0; i < N; ++i) r[i] = b[i] - q[i];
    double nr = norm2_n(N, r);
    double thresh = tol * nb;
    if (reltol * nr > thresh) thresh = reltol * nr;
    *res0_out = nr / nb;
    if (nr <= thresh) goto done;
    amg_vcycle(h, 0, r, z);
    for (int i = 0; i < N; ++i) p[i] = z[i];
    double rho = dot_n(N, r, z);
    for (it = 1; it <= maxit; ++it) {
        ldu_matvec(N, F, own, nei, diag, upper, upper, p, q);
        double pq = dot_n(N, p, q);
        if (!(pq > 0.0) || !isfinite(pq)) { status = -2; break; }
        double alpha = rho / pq;
        for (int i = 0; i < N; ++i) x[i] += alpha * p[i];
        for (int i = 0; i < N; ++i) r[i] -= alpha * q[i];
        nr = norm2_n(N, r);
        if (!isfinite(nr)) { status = -2; break; }
        if (nr <= thresh) break;
        if (it == maxit) { status = -1; break; }
        amg_vcycle(h, 0, r, z);
        double rho_new = dot_n(N, r, z);
        double beta = rho_new / rho;
        rho = rho_new;
        for (int i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
    }
    if (it > maxit) status = -1;
done:
    *res_out = nr / nb;
    *iters_out = it > maxit ? maxit : it;
    free(r); free(z); free(p); free(q);
    return status;
}

/* level-l matrices set by the last V-cycle or solve (tests) */
void orc_amg_matrix(const oamg *h, int l, double *d, double *o)
{
    memcpy(d, h->d[l], sizeof(double) * h->n[l]);
    memcpy(o, h->o[l], sizeof(double) * h->ne[l]);
}

/* edges of level l (tests) */
void orc_amg_edges(const oamg *h, int l, int *ea, int *eb)
{
    memcpy(ea, h->ea[l], sizeof(int) * h->ne[l]);
    memcpy(eb, h->eb[l], sizeof(int) * h->ne[l]);
}
