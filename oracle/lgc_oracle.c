/*
 * FP64 CPU oracle for generalized Laguerre cells -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load this library.  It shares no code with the CUDA path.  It is plain,
 * slow and written to be checked against the paper by eye.
 *
 * What it computes (paper Sec. 2.2 Eq. 1, Sec. 3.1-3.4, Algorithm 2):
 *   C_i = box  intersect  B(p_i, sqrt(psi_i))
 *         intersect_{j != i} { x : |x-p_i|^2 - psi_i <= |x-p_j|^2 - psi_j }.
 *   For every plane f that cuts the ball (bisector with a site j, or a wall):
 *     B_f = (plane facet of the clipped polytope) restricted to the ball (Sec. 3.4)
 *     |B_f|, the signed solid angle Omega_f that B_f subtends at p_i (the
 *     projection of B_f onto the sphere from c = p_i, Sec. 3.3), and
 *     the first moment of B_f.
 *   |K_i| = psi_i * (4 pi [p_i in P_i] - sum_f Omega_f)           (Sec. 3.3)
 *   |V_i| = (1/3) (sum_f h_f |B_f| + sqrt(psi_i) |K_i|)             (Sec. 3.2)
 *   centroid: int_C (x-p) dx = 1/4 sum_f h_f int_{B_f}(x-p) dA
 *                              - 1/4 psi_i sum_f n_f |B_f|
 *
 * Readings of the paper taken here (where it is garbled, ambiguous or silent):
 *   - the pyramid volume is h|B|/3 (the field F=(x-p)/3 of Sec. 3.2 gives the
 *     1/3 that the printed h|B| and sqrt(psi)|K| drop);
 *   - h_f is the scalar signed distance (|d|^2 + psi_i - psi_j) / (2|d|);
 *   - the projection point c of Sec. 3.3 is the site itself, with signed solid
 *     angles and the indicator [p_i inside every half-space], which is exact
 *     whether or not p_i lies in its cell.  The indicator and the signs of
 *     Omega_f come from the same h_f values, so |K| is continuous where a
 *     plane crosses the site.  A plane exactly through the site (h_f == 0) is
 *     moved outward by eta = 2^-40 sqrt(psi_i): the limit of the site moving
 *     into its cell, which stays right when several planes meet at the site
 *     (a site on a box corner); the change in V is O(eta |B_f|);
 *   - a site j can clip C_i only if |p_i - p_j| < r_i + r_j (r = sqrt(max(psi,0))):
 *     on the radical plane x in B_i <=> x in B_j, and farther sites leave B_i
 *     entirely on i's side.  Brute force over all sites is kept as a mode so
 *     tests can check this lemma.
 *
 * Parity pins (tests/test_oracle_*.py): isolated ball, two-ball caps, wall
 * caps, box corner, cubic lattices (two regimes), Monte Carlo volume / free
 * surface / facet areas / centroid, finite differences of V in psi, symmetry
 * of the Hessian, sum of volumes <= box volume, brute force vs grid search.
 *
 * Domain: each polygon vertex is the intersection of two lines, so inputs
 * whose bisector traces are parallel to within about 1e-8 without being
 * identical (a cubic lattice whose float32 positions are off the exact
 * lattice by rounding, or jittered by 1e-5 of the spacing or less,
 * with balls reaching the cube edges) are outside it: there it can return
 * volumes above the lattice cube that contains the cell.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_TOO_MANY_FACETS 1
#define ORC_COINCIDENT 2
#define ORC_MAXV 512

typedef struct { double x, y, z; } v3;

static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 crs(v3 a, v3 b) { return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static double nrm(v3 a) { return sqrt(dot(a, a)); }

/* A cutting plane of cell i: points y (relative to p_i) with y.n = h.
 * kind >= 0: bisector with site `kind` at distance d; kind = -1-w: wall w
 * (w = 0..5 for -x,+x,-y,+y,-z,+z). */
typedef struct { v3 n; double h; double d; int64_t kind; } plane_t;

/* Per-facet results. */
typedef struct { double area, omega; v3 moment; } facet_q;

/* A convex polygon in a facet's plane is kept as the cyclic list of its
 * bounding lines a*x + b*y <= c; vertex k is the intersection of lines k-1
 * and k, always recomputed from the two lines (never interpolated), so a
 * vertex near the foot point keeps its relative precision. */
typedef struct { double a, b, c; } line_t;

static void line_isect(line_t l1, line_t l2, double* x, double* y) {
  double det = l1.a * l2.b - l2.a * l1.b;
  *x = (l1.c * l2.b - l2.c * l1.b) / det;
  *y = (l1.a * l2.c - l2.a * l1.c) / det;
}

/* Clip the polygon (lines L[0..m-1]) by a*x + b*y <= c into out[].
 * Returns the new line count (0 = empty), -1 on overflow. */
static int clip_lines(const line_t* L, int m, line_t nl, line_t* out) {
  int outside[ORC_MAXV];
  int nout = 0;
  for (int k = 0; k < m; k++) {
    double x, y;
    line_isect(L[(k + m - 1) % m], L[k], &x, &y);
    outside[k] = nl.a * x + nl.b * y - nl.c > 0.0;
    nout += outside[k];
  }
  if (nout == 0) { memcpy(out, L, sizeof(line_t) * m); return m; }
  if (nout == m) return 0;
  /* s: first outside vertex after an inside one; e: last of that run */
  int s = -1;
  for (int k = 0; k < m; k++) if (outside[k] && !outside[(k + m - 1) % m]) { s = k; break; }
  int e = s;
  while (outside[(e + 1) % m]) e = (e + 1) % m;
  /* edges s..e-1 lie outside; keep lines e, e+1, ..., s-1, then the new line */
  int no = 0;
  for (int k = e; ; k = (k + 1) % m) {
    out[no++] = L[k];
    if (k == (s + m - 1) % m) break;
  }
  if (no + 1 >= ORC_MAXV) return -1;
  out[no++] = nl;
  return no;
}

/* Orthonormal u, v with u x v = n. */
static void plane_basis(v3 n, v3* u, v3* v) {
  v3 e;
  double ax = fabs(n.x), ay = fabs(n.y), az = fabs(n.z);
  if (ax <= ay && ax <= az) e = mk(1, 0, 0);
  else if (ay <= az) e = mk(0, 1, 0);
  else e = mk(0, 0, 1);
  v3 uu = crs(e, n);
  uu = scl(uu, 1.0 / nrm(uu));
  *u = uu;
  *v = crs(n, uu);
}

/* Solid angle of the triangle (a,b,c) seen from the origin (Van Oosterom &
 * Strackee 1983), signed by the orientation of the triangle. */
static double tri_solid_angle(v3 a, v3 b, v3 c) {
  double la = nrm(a), lb = nrm(b), lc = nrm(c);
  double num = dot(a, crs(b, c));
  double den = la * lb * lc + dot(a, b) * lc + dot(a, c) * lb + dot(b, c) * la;
  return 2.0 * atan2(num, den);
}

/* One piece of the fan of (polygon intersect disk) from the disk centre,
 * in the facet's local frame (s, t, height): the site is the origin, the
 * disk centre is (0,0,h).
 * inside=1: triangle (centre, A, B); inside=0: circular sector of radius rho
 * between the directions of A and B.  Accumulates area, signed solid angle
 * and the in-plane first moment (mx, my) about the disk centre. */
typedef struct { double area, omega, mx, my; } piece_acc;

static void add_piece(piece_acc* q, int inside, double ax, double ay, double bx, double by,
                      double rho, double h, double r) {
  double cr = ax * by - ay * bx;
  double dt = ax * bx + ay * by;
  if (inside) {
    double area = 0.5 * cr;
    double om = tri_solid_angle(mk(0, 0, h), mk(ax, ay, h), mk(bx, by, h));
    q->area += area;
    q->omega += om;
    /* centroid of the triangle (centre, A, B) is (A+B)/3 */
    q->mx += area * (ax + bx) / 3.0;
    q->my += area * (ay + by) / 3.0;
  } else {
    double phi = atan2(cr, dt);
    double area = 0.5 * rho * rho * phi;
    double sg = (h >= 0.0) ? 1.0 : -1.0;
    double om = phi * (sg - h / r);
    double ta = atan2(ay, ax);
    double tb = ta + phi;
    double r3 = rho * rho * rho / 3.0;
    q->area += area;
    q->omega += om;
    q->mx += r3 * (sin(tb) - sin(ta));
    q->my += r3 * (cos(ta) - cos(tb));
  }
}

/* Restrict the convex polygon (lines L[0..m-1]) of plane (n,h) to the disk
 * of radius rho centred at the foot point h*n, and integrate area, solid
 * angle and first moment (3D, about the site). */
static facet_q restrict_polygon(const line_t* L, int m, double rho, double h, double r, v3 n,
                                v3 u, v3 v) {
  facet_q fq;
  piece_acc q = {0.0, 0.0, 0.0, 0.0};
  double xs[ORC_MAXV], ys[ORC_MAXV];
  for (int k = 0; k < m; k++) line_isect(L[(k + m - 1) % m], L[k], &xs[k], &ys[k]);
  double rho2 = rho * rho;
  for (int k = 0; k < m; k++) {
    int k2 = (k + 1 == m) ? 0 : k + 1;
    double px = xs[k], py = ys[k], qx = xs[k2], qy = ys[k2];
    double dx = qx - px, dy = qy - py;
    double a2 = dx * dx + dy * dy;
    if (a2 == 0.0) continue;
    double b2 = px * dx + py * dy;
    double c2 = px * px + py * py - rho2;
    double disc = b2 * b2 - a2 * c2;
    if (disc <= 0.0) {
      add_piece(&q, 0, px, py, qx, qy, rho, h, r);
      continue;
    }
    double sq = sqrt(disc);
    double t1 = (-b2 - sq) / a2, t2 = (-b2 + sq) / a2;
    if (t1 < 0.0) t1 = 0.0;
    if (t1 > 1.0) t1 = 1.0;
    if (t2 < 0.0) t2 = 0.0;
    if (t2 > 1.0) t2 = 1.0;
    /* crossing points; a clamped end is the vertex itself, exactly */
    double x1 = px + t1 * dx, y1 = py + t1 * dy;
    double x2 = px + t2 * dx, y2 = py + t2 * dy;
    if (t1 == 0.0) { x1 = px; y1 = py; }
    if (t1 == 1.0) { x1 = qx; y1 = qy; }
    if (t2 == 0.0) { x2 = px; y2 = py; }
    if (t2 == 1.0) { x2 = qx; y2 = qy; }
    if (t1 > 0.0) add_piece(&q, 0, px, py, x1, y1, rho, h, r);
    if (t2 > t1) add_piece(&q, 1, x1, y1, x2, y2, rho, h, r);
    if (t2 < 1.0) add_piece(&q, 0, x2, y2, qx, qy, rho, h, r);
  }
  fq.area = q.area;
  fq.omega = q.omega;
  fq.moment = add(scl(n, h * q.area), add(scl(u, q.mx), scl(v, q.my)));
  return fq;
}

/* ---------------------------------------------------------------------- */
/* Candidate search: all j != i with |p_i - p_j| < r_i + r_j.               */

typedef struct {
  double lo[3], cs;
  int dim[3];
  int64_t* head;
  int64_t* next;
  double rmax;
} bucket_grid;

static double rad(double psi) { return psi > 0.0 ? sqrt(psi) : 0.0; }

static void grid_build(bucket_grid* g, int64_t n, const double* pos, const double* psi) {
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  double rmax = 0.0;
  for (int64_t i = 0; i < n; i++) {
    for (int k = 0; k < 3; k++) {
      if (pos[3 * i + k] < lo[k]) lo[k] = pos[3 * i + k];
      if (pos[3 * i + k] > hi[k]) hi[k] = pos[3 * i + k];
    }
    if (rad(psi[i]) > rmax) rmax = rad(psi[i]);
  }
  double cs = 2.0 * rmax;
  double ext = 0.0;
  for (int k = 0; k < 3; k++) if (hi[k] - lo[k] > ext) ext = hi[k] - lo[k];
  if (cs < ext / 200.0) cs = ext / 200.0;
  if (cs <= 0.0) cs = 1.0;
  for (int k = 0; k < 3; k++) {
    g->lo[k] = lo[k];
    g->dim[k] = (int)floor((hi[k] - lo[k]) / cs) + 1;
  }
  g->cs = cs;
  g->rmax = rmax;
  int64_t ncell = (int64_t)g->dim[0] * g->dim[1] * g->dim[2];
  g->head = (int64_t*)malloc(sizeof(int64_t) * ncell);
  g->next = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  for (int64_t c = 0; c < ncell; c++) g->head[c] = -1;
  for (int64_t i = n - 1; i >= 0; i--) {
    int c[3];
    for (int k = 0; k < 3; k++) {
      c[k] = (int)floor((pos[3 * i + k] - g->lo[k]) / cs);
      if (c[k] < 0) c[k] = 0;
      if (c[k] >= g->dim[k]) c[k] = g->dim[k] - 1;
    }
    int64_t cid = ((int64_t)c[2] * g->dim[1] + c[1]) * g->dim[0] + c[0];
    g->next[i] = g->head[cid];
    g->head[cid] = i;
  }
}

static void grid_free(bucket_grid* g) { free(g->head); free(g->next); }

/* ---------------------------------------------------------------------- */

typedef struct {
  /* per query */
  double vol, karea, omega_sum;
  v3 cen;
  int inside;    /* [p_i in all half-spaces] */
  int n_planes;  /* cutting planes (walls + bisectors with |h| < r) */
  int status;
} cell_out;

/* Compute one generalized Laguerre cell.  cand: candidate site indices. */
static cell_out one_cell(int64_t i, const double* pos, const double* psi, const double* lo,
                         const double* hi, const int64_t* cand, int ncand, int max_facets,
                         int64_t* fac_j, double* fac_area, double* fac_dist, double* fac_h,
                         int32_t* nfac, double* wall_area, plane_t* pl) {
  cell_out o;
  memset(&o, 0, sizeof(o));
  v3 p = mk(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]);
  o.cen = p;
  *nfac = 0;
  for (int w = 0; w < 6; w++) wall_area[w] = 0.0;
  double ps = psi[i];
  if (!(ps > 0.0)) return o; /* empty cell */
  double r = sqrt(ps);

  /* Gather cutting planes.  Empty cell as soon as one half-space excludes the ball. */
  int np = 0;
  for (int w = 0; w < 6; w++) {
    int ax = w / 2;
    double pk = ax == 0 ? p.x : (ax == 1 ? p.y : p.z);
    double h = (w & 1) ? hi[ax] - pk : pk - lo[ax];
    v3 n = mk(0, 0, 0);
    double sgn = (w & 1) ? 1.0 : -1.0;
    if (ax == 0) n.x = sgn; else if (ax == 1) n.y = sgn; else n.z = sgn;
    if (h == 0.0) h = ldexp(r, -40); /* plane through the site: see header */
    if (h <= -r) { o.vol = 0; o.karea = 0; return o; }
    if (h < r) { pl[np].n = n; pl[np].h = h; pl[np].d = 0; pl[np].kind = -1 - w; np++; }
  }
  for (int c = 0; c < ncand; c++) {
    int64_t j = cand[c];
    v3 dv = sub(mk(pos[3 * j], pos[3 * j + 1], pos[3 * j + 2]), p);
    double d = nrm(dv);
    if (d == 0.0) { o.status = ORC_COINCIDENT; return o; }
    double h = (d * d + ps - psi[j]) / (2.0 * d);
    if (h == 0.0) h = ldexp(r, -40); /* plane through the site: see header */
    if (h <= -r) { o.vol = 0; o.karea = 0; *nfac = 0; return o; }
    if (h < r) { pl[np].n = scl(dv, 1.0 / d); pl[np].h = h; pl[np].d = d; pl[np].kind = j; np++; }
  }
  o.n_planes = np;

  int inside = 1;
  for (int f = 0; f < np; f++) if (pl[f].h < 0.0) inside = 0;
  o.inside = inside;

  double sum_hA = 0.0, sum_om = 0.0;
  v3 sum_hM = mk(0, 0, 0), sum_nA = mk(0, 0, 0);
  int nf = 0;
  for (int f = 0; f < np; f++) {
    v3 n = pl[f].n;
    double h = pl[f].h;
    double rho = sqrt(ps - h * h);
    v3 u, v;
    plane_basis(n, &u, &v);
    /* the facet within a square that contains the disk, clipped by every
     * other plane; only its part inside the disk matters */
    double B = 2.0 * rho;
    line_t la[ORC_MAXV], lb[ORC_MAXV];
    la[0].a = 0; la[0].b = -1; la[0].c = B; /* bottom */
    la[1].a = 1; la[1].b = 0; la[1].c = B;  /* right  */
    la[2].a = 0; la[2].b = 1; la[2].c = B;  /* top    */
    la[3].a = -1; la[3].b = 0; la[3].c = B; /* left   */
    int nl = 4;
    line_t *cur = la, *nxt = lb;
    for (int g = 0; g < np && nl > 0; g++) {
      if (g == f) continue;
      line_t L;
      L.a = dot(u, pl[g].n);
      L.b = dot(v, pl[g].n);
      L.c = pl[g].h - h * dot(n, pl[g].n);
      if (L.a * L.a + L.b * L.b == 0.0) { /* parallel plane: all or nothing */
        if (L.c < 0.0) nl = 0;
        continue;
      }
      int m = clip_lines(cur, nl, L, nxt);
      if (m < 0) { o.status = ORC_TOO_MANY_FACETS; return o; }
      nl = m;
      line_t* t = cur; cur = nxt; nxt = t;
    }
    facet_q q;
    q.area = 0.0; q.omega = 0.0; q.moment = mk(0, 0, 0);
    if (nl >= 3) q = restrict_polygon(cur, nl, rho, h, r, n, u, v);
    sum_hA += h * q.area;
    sum_om += q.omega;
    sum_hM = add(sum_hM, scl(q.moment, h));
    sum_nA = add(sum_nA, scl(n, q.area));
    if (pl[f].kind < 0) {
      wall_area[-1 - pl[f].kind] = q.area;
    } else {
      if (nf >= max_facets) { o.status = ORC_TOO_MANY_FACETS; return o; }
      fac_j[nf] = pl[f].kind;
      fac_area[nf] = q.area;
      fac_dist[nf] = pl[f].d;
      fac_h[nf] = h;
      nf++;
    }
  }
  *nfac = nf;
  double K = ps * (4.0 * M_PI * (double)inside - sum_om);
  if (K < 0.0) K = 0.0;
  o.karea = K;
  o.omega_sum = sum_om;
  o.vol = (sum_hA + r * K) / 3.0;
  if (o.vol > 0.0) {
    v3 m = sub(scl(sum_hM, 0.25), scl(sum_nA, 0.25 * ps));
    o.cen = add(p, scl(m, 1.0 / o.vol));
  }
  return o;
}

/*
 * Batch entry point.
 *   n, pos[n*3], psi[n]: all sites;  lo[3], hi[3]: the box.
 *   nq, query[nq]: indices of the cells to compute.
 *   brute: 1 = test every other site as a candidate, 0 = bucket grid.
 *   max_facets: capacity per query of the facet arrays.
 * Outputs per query q: vol, karea, omega_sum, inside, n_planes, cen[3], status,
 *   wall_area[6], nfac and up to max_facets bisector facets (cutting planes,
 *   area possibly 0): fac_j (site index), fac_area, fac_dist, fac_h.
 * Returns the number of queries whose status is not 0.
 */
int oracle_cells(int64_t n, const double* pos, const double* psi, const double* lo,
                 const double* hi, int64_t nq, const int64_t* query, int brute, int max_facets,
                 double* vol, double* karea, double* omega_sum, int32_t* inside,
                 int32_t* n_planes, double* cen, int32_t* status, double* wall_area,
                 int32_t* nfac, int64_t* fac_j, double* fac_area, double* fac_dist,
                 double* fac_h, int nthreads) {
  bucket_grid g;
  memset(&g, 0, sizeof(g));
  if (!brute) grid_build(&g, n, pos, psi);
  int nbad = 0;
  /* the thread count applies to this call only (a num_threads clause, not
     the process-wide setting, so a later call with 0 gets every core again) */
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  int nt = 1;
#endif
  (void)nt;
#pragma omp parallel num_threads(nt) reduction(+ : nbad)
  {
    int64_t cap = brute ? (n > 0 ? n : 1) : 4096;
    int64_t* cand = (int64_t*)malloc(sizeof(int64_t) * cap);
    plane_t* pl = (plane_t*)malloc(sizeof(plane_t) * (cap + 6));
#pragma omp for schedule(dynamic, 16)
    for (int64_t q = 0; q < nq; q++) {
      int64_t i = query[q];
      double ri = rad(psi[i]);
      int nc = 0;
      int over = 0;
      if (brute) {
        for (int64_t j = 0; j < n; j++) {
          if (j == i) continue;
          double dx = pos[3 * j] - pos[3 * i], dy = pos[3 * j + 1] - pos[3 * i + 1],
                 dz = pos[3 * j + 2] - pos[3 * i + 2];
          double d = sqrt(dx * dx + dy * dy + dz * dz);
          if (d < ri + rad(psi[j])) cand[nc++] = j;
        }
      } else if (ri > 0.0) {
        double R = ri + g.rmax;
        int c0[3], c1[3];
        for (int k = 0; k < 3; k++) {
          c0[k] = (int)floor((pos[3 * i + k] - R - g.lo[k]) / g.cs);
          c1[k] = (int)floor((pos[3 * i + k] + R - g.lo[k]) / g.cs);
          if (c0[k] < 0) c0[k] = 0;
          if (c1[k] >= g.dim[k]) c1[k] = g.dim[k] - 1;
        }
        for (int cz = c0[2]; cz <= c1[2]; cz++)
          for (int cy = c0[1]; cy <= c1[1]; cy++)
            for (int cx = c0[0]; cx <= c1[0]; cx++) {
              int64_t cid = ((int64_t)cz * g.dim[1] + cy) * g.dim[0] + cx;
              for (int64_t j = g.head[cid]; j >= 0; j = g.next[j]) {
                if (j == i) continue;
                double dx = pos[3 * j] - pos[3 * i], dy = pos[3 * j + 1] - pos[3 * i + 1],
                       dz = pos[3 * j + 2] - pos[3 * i + 2];
                double d = sqrt(dx * dx + dy * dy + dz * dz);
                if (d < ri + rad(psi[j])) {
                  if (nc >= cap) { over = 1; continue; }
                  cand[nc++] = j;
                }
              }
            }
      }
      cell_out o;
      if (over) {
        memset(&o, 0, sizeof(o));
        o.status = ORC_TOO_MANY_FACETS;
        nfac[q] = 0;
      } else {
        o = one_cell(i, pos, psi, lo, hi, cand, nc, max_facets, fac_j + q * max_facets,
                     fac_area + q * max_facets, fac_dist + q * max_facets,
                     fac_h + q * max_facets, nfac + q, wall_area + 6 * q, pl);
      }
      vol[q] = o.vol;
      karea[q] = o.karea;
      omega_sum[q] = o.omega_sum;
      inside[q] = o.inside;
      n_planes[q] = o.n_planes;
      cen[3 * q] = o.cen.x;
      cen[3 * q + 1] = o.cen.y;
      cen[3 * q + 2] = o.cen.z;
      status[q] = o.status;
      if (o.status) nbad++;
    }
    free(cand);
    free(pl);
  }
  if (!brute) grid_free(&g);
  return nbad;
}

/* Number of OpenMP threads the library would use (1 without OpenMP). */
int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
