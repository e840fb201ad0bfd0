/*
 * CPU oracle -- TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and
 * the CPU-baseline leg of the benchmark may load this library; the product
 * path never does.  It shares no code with the CUDA library.
 *
 * Contents
 *   1. Exact orientation / in-circle signs for arbitrary doubles, by floating
 *      expansion arithmetic (Shewchuk 1997, "Adaptive precision floating-point
 *      arithmetic and fast robust geometric predicates"): every determinant is
 *      evaluated as a non-overlapping expansion whose largest component gives
 *      the exact sign.  A plain double evaluation with a conservative error
 *      bound answers the easy cases first.
 *   2. A Delaunay triangulation of the disk centres plus four fixed corner
 *      points, built from scratch by Bowyer-Watson insertion.  The paper
 *      builds its initial triangulation once on the host (Sec. 4.1); the
 *      oracle rebuilds it from scratch whenever it needs the triangulation of
 *      new positions, so it never depends on edge flips.
 *   3. Direct O(N^2) sums of the long-range pair force of Sec. 2.2 in FP64.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC
 * (-ffp-contract=off keeps the compiler from fusing the two-sum steps).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* 1. expansion arithmetic                                             */
/* ------------------------------------------------------------------ */

static void two_sum(double a, double b, double *x, double *y) {
    double s = a + b;
    double bv = s - a;
    double av = s - bv;
    *x = s;
    *y = (a - av) + (b - bv);
}

static void two_prod(double a, double b, double *x, double *y) {
    double p = a * b;
    *x = p;
    *y = fma(a, b, -p); /* exact low part of a*b */
}

/* h = e + b, e non-overlapping increasing; returns length (zeros dropped) */
static int grow_expansion(int elen, const double *e, double b, double *h) {
    double q = b, qn, hh;
    int k = 0;
    for (int i = 0; i < elen; i++) {
        two_sum(q, e[i], &qn, &hh);
        q = qn;
        if (hh != 0.0) h[k++] = hh;
    }
    if (q != 0.0 || k == 0) h[k++] = q;
    return k;
}

/* h = e + f by repeated growth; h must not alias e or f */
static int expansion_sum(int elen, const double *e, int flen, const double *f, double *h) {
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(elen + flen + 1));
    int hl = elen;
    memcpy(h, e, sizeof(double) * (size_t)elen);
    for (int j = 0; j < flen; j++) {
        hl = grow_expansion(hl, h, f[j], tmp);
        memcpy(h, tmp, sizeof(double) * (size_t)hl);
    }
    free(tmp);
    return hl;
}

/* h = e * b */
static int scale_expansion(int elen, const double *e, double b, double *h) {
    /* every e[i]*b is exactly p1+p0; add them all in by growth */
    int hl = 1;
    h[0] = 0.0;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(2 * elen + 2));
    for (int i = 0; i < elen; i++) {
        double p1, p0;
        two_prod(e[i], b, &p1, &p0);
        hl = grow_expansion(hl, h, p0, tmp);
        memcpy(h, tmp, sizeof(double) * (size_t)hl);
        hl = grow_expansion(hl, h, p1, tmp);
        memcpy(h, tmp, sizeof(double) * (size_t)hl);
    }
    free(tmp);
    return hl;
}

/* h = e * f */
static int mul_expansion(int elen, const double *e, int flen, const double *f, double *h) {
    double *part = (double *)malloc(sizeof(double) * (size_t)(2 * elen + 2));
    size_t cap = (size_t)(2 * elen + 1) * (size_t)flen + 2;
    double *acc = (double *)malloc(sizeof(double) * cap);
    double *tmp = (double *)malloc(sizeof(double) * cap);
    int al = 1;
    acc[0] = 0.0;
    for (int j = 0; j < flen; j++) {
        int pl = scale_expansion(elen, e, f[j], part);
        al = expansion_sum(al, acc, pl, part, tmp);
        memcpy(acc, tmp, sizeof(double) * (size_t)al);
    }
    memcpy(h, acc, sizeof(double) * (size_t)al);
    free(part);
    free(acc);
    free(tmp);
    return al;
}

static int neg_expansion(int elen, const double *e, double *h) {
    for (int i = 0; i < elen; i++) h[i] = -e[i];
    return elen;
}

static int sign_expansion(int elen, const double *e) {
    double top = e[elen - 1];
    return (top > 0.0) - (top < 0.0);
}

/* exact a - b as a two-component expansion */
static int diff2(double a, double b, double *h) {
    double x, y;
    two_sum(a, -b, &x, &y);
    h[0] = y;
    h[1] = x;
    return 2;
}

/* exact sign of (bx-ax)(cy-ay) - (by-ay)(cx-ax): >0 iff a,b,c counter-clockwise */
int oracle_orient2d_exact(double ax, double ay, double bx, double by, double cx, double cy) {
    double bax[2], bay[2], cax[2], cay[2];
    diff2(bx, ax, bax);
    diff2(by, ay, bay);
    diff2(cx, ax, cax);
    diff2(cy, ay, cay);
    double t1[16], t2[16], nt2[16], det[40];
    int l1 = mul_expansion(2, bax, 2, cay, t1);
    int l2 = mul_expansion(2, bay, 2, cax, t2);
    neg_expansion(l2, t2, nt2);
    int ld = expansion_sum(l1, t1, l2, nt2, det);
    return sign_expansion(ld, det);
}

int oracle_orient2d(double ax, double ay, double bx, double by, double cx, double cy) {
    double l = (bx - ax) * (cy - ay);
    double r = (by - ay) * (cx - ax);
    double det = l - r;
    double bound = 1e-14 * (fabs(l) + fabs(r));
    if (det > bound) return 1;
    if (-det > bound) return -1;
    return oracle_orient2d_exact(ax, ay, bx, by, cx, cy);
}

/* exact sign of the in-circle determinant: >0 iff d lies strictly inside the
 * circle through a, b, c (given counter-clockwise) */
int oracle_incircle_exact(double ax, double ay, double bx, double by, double cx, double cy,
                          double dx, double dy) {
    double adx[2], ady[2], bdx[2], bdy[2], cdx[2], cdy[2];
    diff2(ax, dx, adx);
    diff2(ay, dy, ady);
    diff2(bx, dx, bdx);
    diff2(by, dy, bdy);
    diff2(cx, dx, cdx);
    diff2(cy, dy, cdy);
    /* lifts */
    double s1[16], s2[16], alift[40], blift[40], clift[40];
    int la, lb, lc, l1, l2;
    l1 = mul_expansion(2, adx, 2, adx, s1);
    l2 = mul_expansion(2, ady, 2, ady, s2);
    la = expansion_sum(l1, s1, l2, s2, alift);
    l1 = mul_expansion(2, bdx, 2, bdx, s1);
    l2 = mul_expansion(2, bdy, 2, bdy, s2);
    lb = expansion_sum(l1, s1, l2, s2, blift);
    l1 = mul_expansion(2, cdx, 2, cdx, s1);
    l2 = mul_expansion(2, cdy, 2, cdy, s2);
    lc = expansion_sum(l1, s1, l2, s2, clift);
    /* 2x2 minors */
    double m1[16], m2[16], nm2[16], bc[40], ca[40], ab[40];
    int lbc, lca, lab;
    l1 = mul_expansion(2, bdx, 2, cdy, m1);
    l2 = mul_expansion(2, bdy, 2, cdx, m2);
    neg_expansion(l2, m2, nm2);
    lbc = expansion_sum(l1, m1, l2, nm2, bc);
    l1 = mul_expansion(2, cdx, 2, ady, m1);
    l2 = mul_expansion(2, cdy, 2, adx, m2);
    neg_expansion(l2, m2, nm2);
    lca = expansion_sum(l1, m1, l2, nm2, ca);
    l1 = mul_expansion(2, adx, 2, bdy, m1);
    l2 = mul_expansion(2, ady, 2, bdx, m2);
    neg_expansion(l2, m2, nm2);
    lab = expansion_sum(l1, m1, l2, nm2, ab);
    /* alift*bc + blift*ca + clift*ab */
    size_t cap = (size_t)(81 * 40 + 8);
    double *ta = (double *)malloc(sizeof(double) * cap);
    double *tb = (double *)malloc(sizeof(double) * cap);
    double *tc = (double *)malloc(sizeof(double) * cap);
    double *u = (double *)malloc(sizeof(double) * 2 * cap);
    double *det = (double *)malloc(sizeof(double) * 3 * cap);
    int lta = mul_expansion(la, alift, lbc, bc, ta);
    int ltb = mul_expansion(lb, blift, lca, ca, tb);
    int ltc = mul_expansion(lc, clift, lab, ab, tc);
    int lu = expansion_sum(lta, ta, ltb, tb, u);
    int ld = expansion_sum(lu, u, ltc, tc, det);
    int s = sign_expansion(ld, det);
    free(ta);
    free(tb);
    free(tc);
    free(u);
    free(det);
    return s;
}

int oracle_incircle(double ax, double ay, double bx, double by, double cx, double cy,
                    double dx, double dy) {
    double adx = ax - dx, ady = ay - dy;
    double bdx = bx - dx, bdy = by - dy;
    double cdx = cx - dx, cdy = cy - dy;
    double bc = bdx * cdy - bdy * cdx;
    double ca = cdx * ady - cdy * adx;
    double ab = adx * bdy - ady * bdx;
    double al = adx * adx + ady * ady;
    double bl = bdx * bdx + bdy * bdy;
    double cl = cdx * cdx + cdy * cdy;
    double det = al * bc + bl * ca + cl * ab;
    double perm = al * (fabs(bdx * cdy) + fabs(bdy * cdx)) + bl * (fabs(cdx * ady) + fabs(cdy * adx)) +
                  cl * (fabs(adx * bdy) + fabs(ady * bdx));
    double bound = 1e-14 * perm;
    if (det > bound) return 1;
    if (-det > bound) return -1;
    return oracle_incircle_exact(ax, ay, bx, by, cx, cy, dx, dy);
}

/* ------------------------------------------------------------------ */
/* 2. Bowyer-Watson Delaunay triangulation                              */
/* ------------------------------------------------------------------ */

typedef struct {
    const double *x, *y;
    int *tv;    /* 3 vertices per triangle, counter-clockwise */
    int *tn;    /* neighbour across the edge opposite vertex k, -1 = none */
    char *alive;
    int ntri, cap;
    int *freelist;
    int nfree;
} mesh_t;

static int new_tri(mesh_t *m) {
    if (m->nfree > 0) return m->freelist[--m->nfree];
    return m->ntri++;
}

static int in_circle_tri(const mesh_t *m, int t, double px, double py) {
    const int *v = m->tv + 3 * t;
    return oracle_incircle(m->x[v[0]], m->y[v[0]], m->x[v[1]], m->y[v[1]], m->x[v[2]], m->y[v[2]], px,
                           py);
}

/* Walk from triangle t to a triangle containing point p (inside or on its boundary). */
static int locate(const mesh_t *m, int t, double px, double py, int *steps_out) {
    int steps = 0;
    int rot = 0;
    for (;;) {
        const int *v = m->tv + 3 * t;
        int moved = 0;
        for (int kk = 0; kk < 3; kk++) {
            int k = (kk + rot) % 3;
            int a = v[(k + 1) % 3], b = v[(k + 2) % 3];
            if (oracle_orient2d(m->x[a], m->y[a], m->x[b], m->y[b], px, py) < 0) {
                int nb = m->tn[3 * t + k];
                if (nb < 0) return -1; /* outside the hull */
                t = nb;
                moved = 1;
                break;
            }
        }
        rot = (rot + 1) % 3;
        steps++;
        if (!moved) break;
        if (steps > 100000000) return -2;
    }
    if (steps_out) *steps_out = steps;
    return t;
}

/*
 * Delaunay triangulation of n points (x[i], y[i]) inserted in the order given
 * by `order` (a permutation of 0..n-1; any order gives the same result for
 * points in general position), inside the square with corners
 * (x[n..n+3], y[n..n+3]) which must enclose every point strictly and be given
 * counter-clockwise.  Writes 3 vertex ids per triangle (counter-clockwise) to
 * tri_out (capacity 3*(2n+2)) and returns the number of triangles, or a
 * negative code (-1 point outside, -2 duplicate point, -3 internal error).
 */
int oracle_delaunay(int n, const double *x, const double *y, const int *order, int *tri_out) {
    mesh_t m;
    int cap = 2 * n + 64;
    m.x = x;
    m.y = y;
    m.tv = (int *)malloc(sizeof(int) * 3 * (size_t)cap);
    m.tn = (int *)malloc(sizeof(int) * 3 * (size_t)cap);
    m.alive = (char *)calloc((size_t)cap, 1);
    m.freelist = (int *)malloc(sizeof(int) * (size_t)cap);
    m.nfree = 0;
    m.ntri = 0;
    m.cap = cap;
    int g0 = n, g1 = n + 1, g2 = n + 2, g3 = n + 3;
    /* two triangles of the corner square */
    int t0 = new_tri(&m), t1 = new_tri(&m);
    m.tv[3 * t0 + 0] = g0; m.tv[3 * t0 + 1] = g1; m.tv[3 * t0 + 2] = g2;
    m.tv[3 * t1 + 0] = g0; m.tv[3 * t1 + 1] = g2; m.tv[3 * t1 + 2] = g3;
    /* t0: edge opposite g0 = (g1,g2) hull; opposite g1 = (g2,g0) shared; opposite g2 = (g0,g1) hull */
    m.tn[3 * t0 + 0] = -1; m.tn[3 * t0 + 1] = t1; m.tn[3 * t0 + 2] = -1;
    /* t1: opposite g0 = (g2,g3) hull; opposite g2 = (g3,g0) hull; opposite g3 = (g0,g2) shared */
    m.tn[3 * t1 + 0] = -1; m.tn[3 * t1 + 1] = -1; m.tn[3 * t1 + 2] = t0;
    m.alive[t0] = m.alive[t1] = 1;

    int *stack = (int *)malloc(sizeof(int) * (size_t)cap);
    char *incav = (char *)calloc((size_t)cap, 1);
    int *cav = (int *)malloc(sizeof(int) * (size_t)cap);
    int bcap = 1024;
    int *bu = (int *)malloc(sizeof(int) * bcap), *bv = (int *)malloc(sizeof(int) * bcap),
        *bout = (int *)malloc(sizeof(int) * bcap), *bnew = (int *)malloc(sizeof(int) * bcap);
    int last = t0;
    int rc = 0;
    for (int ii = 0; ii < n && rc == 0; ii++) {
        int p = order[ii];
        double px = x[p], py = y[p];
        int t = locate(&m, last, px, py, NULL);
        if (t < 0) { rc = -1; break; }
        /* duplicate check */
        for (int k = 0; k < 3; k++) {
            int v = m.tv[3 * t + k];
            if (x[v] == px && y[v] == py) rc = -2;
        }
        if (rc) break;
        /* cavity: triangles whose circumcircle strictly contains p, grown from t */
        int ncav = 0, sp = 0;
        stack[sp++] = t;
        incav[t] = 1;
        while (sp > 0) {
            int c = stack[--sp];
            cav[ncav++] = c;
            for (int k = 0; k < 3; k++) {
                int nb = m.tn[3 * c + k];
                if (nb >= 0 && !incav[nb] && in_circle_tri(&m, nb, px, py) > 0) {
                    incav[nb] = 1;
                    stack[sp++] = nb;
                }
            }
        }
        /* boundary edges of the cavity */
        int nb_ = 0;
        for (int q = 0; q < ncav; q++) {
            int c = cav[q];
            for (int k = 0; k < 3; k++) {
                int nb = m.tn[3 * c + k];
                if (nb >= 0 && incav[nb]) continue;
                if (nb_ >= bcap) {
                    bcap *= 2;
                    bu = (int *)realloc(bu, sizeof(int) * bcap);
                    bv = (int *)realloc(bv, sizeof(int) * bcap);
                    bout = (int *)realloc(bout, sizeof(int) * bcap);
                    bnew = (int *)realloc(bnew, sizeof(int) * bcap);
                }
                bu[nb_] = m.tv[3 * c + (k + 1) % 3];
                bv[nb_] = m.tv[3 * c + (k + 2) % 3];
                bout[nb_] = nb;
                nb_++;
            }
        }
        for (int q = 0; q < ncav; q++) {
            incav[cav[q]] = 0;
            m.alive[cav[q]] = 0;
            m.freelist[m.nfree++] = cav[q];
        }
        /* fan of new triangles (u, v, p) */
        for (int e = 0; e < nb_; e++) {
            int nt = new_tri(&m);
            if (nt >= cap) { rc = -3; break; }
            bnew[e] = nt;
            m.alive[nt] = 1;
            m.tv[3 * nt + 0] = bu[e];
            m.tv[3 * nt + 1] = bv[e];
            m.tv[3 * nt + 2] = p;
            m.tn[3 * nt + 2] = bout[e];
            if (bout[e] >= 0) {
                /* point the outside neighbour back at the new triangle */
                int o = bout[e];
                for (int k = 0; k < 3; k++) {
                    int a = m.tv[3 * o + (k + 1) % 3], b = m.tv[3 * o + (k + 2) % 3];
                    if (a == bv[e] && b == bu[e]) m.tn[3 * o + k] = nt;
                }
            }
        }
        if (rc) break;
        /* links between fan triangles: (u,v,p) shares (v,p) with the fan
         * triangle starting at v and (p,u) with the one ending at u */
        for (int e = 0; e < nb_; e++) {
            int nt = bnew[e];
            int found_v = 0, found_u = 0;
            for (int f = 0; f < nb_; f++) {
                if (bu[f] == bv[e]) { m.tn[3 * nt + 0] = bnew[f]; found_v = 1; }
                if (bv[f] == bu[e]) { m.tn[3 * nt + 1] = bnew[f]; found_u = 1; }
            }
            if (!found_v || !found_u) { rc = -3; break; }
        }
        last = bnew[0];
    }
    int nt_out = 0;
    if (rc == 0) {
        for (int t = 0; t < m.ntri; t++) {
            if (!m.alive[t]) continue;
            tri_out[3 * nt_out + 0] = m.tv[3 * t + 0];
            tri_out[3 * nt_out + 1] = m.tv[3 * t + 1];
            tri_out[3 * nt_out + 2] = m.tv[3 * t + 2];
            nt_out++;
        }
    }
    free(m.tv); free(m.tn); free(m.alive); free(m.freelist);
    free(stack); free(incav); free(cav); free(bu); free(bv); free(bout); free(bnew);
    return rc ? rc : nt_out;
}

/* ------------------------------------------------------------------ */
/* 3. direct long-range pair force, Sec. 2.2                            */
/* ------------------------------------------------------------------ */

/* F_i = sum_{j != i} A[s_i][s_j] (r_i - r_j) / |r_i - r_j|^3 for i in [i0, i1) */
void oracle_force_long(int n, const double *x, const double *y, const uint8_t *s, const double *A,
                       int ns, int i0, int i1, double *fx, double *fy, int nthreads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int i = i0; i < i1; i++) {
        double ax = 0.0, ay = 0.0;
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            double rx = x[i] - x[j], ry = y[i] - y[j];
            double r2 = rx * rx + ry * ry;
            double r = sqrt(r2);
            double c = A[ns * s[i] + s[j]] / (r2 * r);
            ax += c * rx;
            ay += c * ry;
        }
        fx[i - i0] = ax;
        fy[i - i0] = ay;
    }
    (void)nthreads;
}

/* The same sum in a periodic box of side L with the minimum-image
 * convention (Sec. 2.1): r_ij is replaced by its image nearest the origin,
 * r_ij - L round(r_ij / L) per component. */
void oracle_force_long_periodic(int n, const double *x, const double *y, const uint8_t *s,
                                const double *A, int ns, double L, int i0, int i1, double *fx,
                                double *fy, int nthreads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int i = i0; i < i1; i++) {
        double ax = 0.0, ay = 0.0;
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            double rx = x[i] - x[j], ry = y[i] - y[j];
            rx -= L * nearbyint(rx / L);
            ry -= L * nearbyint(ry / L);
            double r2 = rx * rx + ry * ry;
            double r = sqrt(r2);
            double c = A[ns * s[i] + s[j]] / (r2 * r);
            ax += c * rx;
            ay += c * ry;
        }
        fx[i - i0] = ax;
        fy[i - i0] = ay;
    }
    (void)nthreads;
}

/* Derivatives of the long-range force F_i = sum_j A[s_i][s_j] r_ij/|r_ij|^3,
 * r_ij = r_i - r_j (Sec. 2.2), for the differentiated rollout.
 *
 * oracle_force_long_jvp: K directions t (tx[k*n + i], ty[k*n + i]); out
 * receives (dF/dx) t, i.e. for every i
 *   sum_j A[s_i][s_j] M(r_ij) (t_i - t_j),   M(r) = I/|r|^3 - 3 r r^T/|r|^5,
 * the derivative of r/|r|^3 with respect to r. */
void oracle_force_long_jvp(int n, const double *x, const double *y, const uint8_t *s, const double *A,
                           int K, const double *tx, const double *ty, double *ox, double *oy,
                           int nthreads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int i = 0; i < n; i++) {
        for (int k = 0; k < K; k++) {
            double ax = 0.0, ay = 0.0;
            const double *txk = tx + (size_t)k * n, *tyk = ty + (size_t)k * n;
            for (int j = 0; j < n; j++) {
                if (j == i) continue;
                double rx = x[i] - x[j], ry = y[i] - y[j];
                double r2 = rx * rx + ry * ry;
                double r = sqrt(r2);
                double r3 = r2 * r, r5 = r3 * r2;
                double dx = txk[i] - txk[j], dy = tyk[i] - tyk[j];
                double c = A[2 * s[i] + s[j]];
                /* M (dx, dy) */
                double mx = dx / r3 - 3.0 * rx * (rx * dx + ry * dy) / r5;
                double my = dy / r3 - 3.0 * ry * (rx * dx + ry * dy) / r5;
                ax += c * mx;
                ay += c * my;
            }
            ox[(size_t)k * n + i] = ax;
            oy[(size_t)k * n + i] = ay;
        }
    }
    (void)nthreads;
}

/* oracle_force_long_dA: S[i][b] = sum over j != i with s_j = b of r_ij/|r_ij|^3,
 * stored as S[4*i + 2*b + 0] (x) and S[4*i + 2*b + 1] (y); then
 * dF_i/dA[a][b] = S[i][b] when s_i = a, else 0. */
void oracle_force_long_dA(int n, const double *x, const double *y, const uint8_t *s, double *S,
                          int nthreads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int i = 0; i < n; i++) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            double rx = x[i] - x[j], ry = y[i] - y[j];
            double r2 = rx * rx + ry * ry;
            double r = sqrt(r2);
            int b = s[j] ? 1 : 0;
            acc[2 * b] += rx / (r2 * r);
            acc[2 * b + 1] += ry / (r2 * r);
        }
        for (int q = 0; q < 4; q++) S[4 * i + q] = acc[q];
    }
    (void)nthreads;
}

int oracle_has_openmp(void) {
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}
