// Generalized Laguerre cells on the GPU (Eq. 1, Sec. 3.2-3.4, Algorithm 2).
//
// Two kernels per evaluation, both in grid-sorted order:
//
// k_candidates (one thread per cell): exact query over the grid around p_i.
//   Site j is kept iff its radical plane cuts the ball of i (|h_ij| < r_i,
//   which implies |p_i - p_j| < r_i + r_j) and lies within the cell's
//   security radius (h_ij < R_i, see below); a plane with h <= -r_i empties
//   the cell.  The six box walls are planes too.
//
// k_cells (one warp per group of 32 cells, one lane per (cell, plane) slot):
//   the planes of consecutive cells fill a shared buffer, and their slots are
//   evaluated 32 per round.  Lane f clips the disk of its plane f by the
//   traces of the other planes of its cell (2D convex clipping of a
//   line-list polygon: every vertex is recomputed from its two lines, never
//   interpolated), restricts the polygon to the disk (Sec. 3.4)
//   and integrates, per fan piece from the disk centre, the facet area
//   |B_f|, the signed solid angle Omega_f it subtends at the site (its
//   projection on the sphere, Sec. 3.3) and its first moment.  Segmented
//   warp reductions then give per cell
//     |K_i| = psi_i (4 pi [p_i inside all planes] - sum_f Omega_f)
//             (0 when no facet reaches the sphere),
//     |V_i| = (sum_f h_f |B_f| + r_i |K_i|) / 3          (pyramids, Sec. 3.2),
//     centroid, and the Hessian row of Eq. 2 (M = -grad^2 K):
//     M_ij = -|B_ij|/(2 d_ij), M_ii = sum_j |B_ij|/(2 d_ij) + |K_i|/(2 r_i).
//   The paper's interior point c (Sec. 3.3) is replaced by the site with
//   signed solid angles, exact whether or not p_i lies in its cell.
#include <math.h>

#include <algorithm>

#include "pot_internal.cuh"

namespace pot {
namespace {

template <typename T>
__device__ __forceinline__ T sqdist(const V4<T>& pi, const V4<T>& pj, T& dx, T& dy, T& dz) {
  dx = r_sub(pj.x, pi.x);
  dy = r_sub(pj.y, pi.y);
  dz = r_sub(pj.z, pi.z);
  return r_add(r_add(r_mul(dx, dx), r_mul(dy, dy)), r_mul(dz, dz));
}

// offset of the radical plane: h = (d^2 + psi_i - psi_j) / (2 d)
template <typename T>
__device__ __forceinline__ T plane_offset(T d2, T psi_i, T psi_j, T& d) {
  d = r_sqrt(d2);
  return r_div(r_add(d2, r_sub(psi_i, psi_j)), r_add(d, d));
}

template <typename T>
__device__ __forceinline__ int cell_coord(T x, T lo, T inv_cs, int dim) {
  T f = (x - lo) * inv_cs;
  int c = (f < T(0)) ? 0 : (f >= T(dim) ? dim - 1 : (int)f);
  return c;
}

__device__ __forceinline__ void set_error(int32_t* err, int code, int64_t site) {
  atomicMax(&err[kErrCode], code);
  atomicMin(&err[kErrSite], (int)site);
}

// ---------------------------------------------------------------------------
// candidates

// Security ball (the paper's contributing-neighbour problem, Sec. 4): a cell
// is built from the bisectors that meet the ball of radius R_i around
// p_i + o_i only (signed distance of the plane from that centre,
// h_ij - n_ij . o_i, below R_i).  If the cell so built lies strictly inside
// that ball, no other plane can touch it and the cell is exact; otherwise
// R_i grows and the cell is rebuilt (pass loop in cells_eval).  Inside deep
// fluid the weights grow like a pressure and the balls get many spacings
// wide, while the cells stay small, and off their sites: centred on the
// cell (o_i = the previous centroid - p_i), the ball keeps the candidate
// lists short.  R_i >= r_i + |o_i| contains the site's ball: every plane
// that cuts it is then a candidate.
//
// The first R_i of an evaluation is a guess from the previous evaluation's
// cells, and a growth step can overshoot (a cell built from too few planes
// can look almost as wide as its ball), so a list that overflows k_max does
// not yet mean the cell needs more than k_max planes.  Each cell keeps a
// bracket: R_lo, the largest radius at which its cell was built and found
// too small, and the current R_i.  An overflow at R_i retries at the
// midpoint of (R_lo, R_i) (R_i / 2 while R_lo = 0); only when the bracket has
// narrowed to 3 % of R_i is the overflow a real capacity error.  A list of
// more than kPlaneCap planes is bisected the same way (a smaller radius may
// still give a short list), and only when its bracket has collapsed does the
// cell keep that many; from then on (for the rest of the evaluation) it grows
// without that limit.  Cells of more than kSmallPlanes planes go to the
// big-cell kernel.
//
// Per-site neighbour lists of the candidate pass (kVerletCap sorted indices
// per site, their count and the reach they were built with; reach 0: none).
template <typename T>
struct VerletList {
  int32_t* list;
  int32_t* count;
  T* reach;
};

// Largest weight near a site: the grid's cells grouped f x f x f into coarse
// cells, and per coarse cell the largest weight over its 3 x 3 x 3 coarse
// neighbourhood (nb == nullptr: not formed; the global largest weight
// serves).  A site j outside the neighbourhood of p_i's coarse cell differs
// from it by more than f fine cells along some axis, so it lies farther
// than (f - 1/2) cs from p_i (the half cell covers the rounding of the cell
// coordinates).
template <typename T>
struct Coarse {
  const T* nb;
  int f;
  int dim[3];
};

template <typename T>
__device__ __forceinline__ int64_t coarse_key(const V4<T>& p, const GridParams<T>& g,
                                              const Coarse<T>& co) {
  // (clamped: a coordinate that is not a number stays inside the grid)
  const int cx = min(max(cell_coord(p.x, g.lo[0], g.inv_cs, g.dim[0]) / co.f, 0), co.dim[0] - 1);
  const int cy = min(max(cell_coord(p.y, g.lo[1], g.inv_cs, g.dim[1]) / co.f, 0), co.dim[1] - 1);
  const int cz = min(max(cell_coord(p.z, g.lo[2], g.inv_cs, g.dim[2]) / co.f, 0), co.dim[2] - 1);
  return ((int64_t)cz * co.dim[1] + cy) * co.dim[0] + cx;
}

template <typename T>
__global__ void __launch_bounds__(256)
    k_candidates(int64_t n, const V4<T>* __restrict__ sxp, const int32_t* __restrict__ cell_start,
                 GridParams<T> g, Box<T> box, const T* __restrict__ psi_max,
                 T* __restrict__ srad, const T* __restrict__ srad_lo,
                 const T* __restrict__ soff, uint8_t* __restrict__ need, int kmax,
                 int32_t* __restrict__ cand, int32_t* __restrict__ meta, int32_t* big_count,
                 int32_t* big_list, int32_t* err, VerletList<T> vl, Coarse<T> co) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n || !need[s]) return;
  const V4<T> p = sxp[s];
  const T ps = p.w;
  if (!(ps > T(0))) {
    meta[s] = kMetaEmpty;
    return;
  }
  const T r = r_sqrt(ps);
  int wmask = 0, nw = 0;
  for (int w = 0; w < 6; w++) {
    T h = fix_zero(wall_offset(p, w, box.lo, box.hi), r);
    if (h <= -r) {
      meta[s] = kMetaEmpty;
      return;
    }
    if (h < r) {
      wmask |= 1 << w;
      nw++;
    }
  }
  const T R = srad[s];
  const T ox = soff[3 * s + 0], oy = soff[3 * s + 1], oz = soff[3 * s + 2];
  // a candidate has h_ij < R + |o| =: Re, so it lies within
  // Re + sqrt(Re^2 - psi_i + psi_j) of p_i, and one that cuts the ball
  // within r + r_j
  const T Re = R + sqrt(ox * ox + oy * oy + oz * oz);
  const T pmx = *psi_max;
  T D = fmin(Re + sqrt(fmax(Re * Re - ps + pmx, T(0))), r + sqrt(pmx));
  // With the global largest weight, no site beyond D is a candidate.  When
  // D stays within the coarse neighbourhood's reach, the sites beyond that
  // reach are excluded by the same bound, and those inside it carry at most
  // the neighbourhood's largest weight, which gives the same bound with a
  // smaller weight.
  if (co.nb != nullptr && D <= (T(co.f) - T(0.5)) * g.cs) {
    const T pl = co.nb[coarse_key(p, g, co)];
    D = fmin(D, fmin(Re + sqrt(fmax(Re * Re - ps + pl, T(0))), r + sqrt(pl)));
  }
  // The bound holds in exact arithmetic; a site right at it (a plane that
  // only touches the ball, or lies on the security ball) is left to the
  // tests on h below, which decide it in their own rounding: the reach
  // carries a relative margin far above the rounding of D and of d.
  D *= T(1.0001);
  const T D2 = D * D;
  int nc = 0;
  bool empty = false;
  const int64_t row = s * (int64_t)kmax;
  // the tests of one site t within the reach D: beyond it no plane can be
  // a candidate or empty the cell; within it the tests on h decide (h < r
  // needs |p_i - p_j| < r_i + r_j, and h <= -r needs p_i inside ball j)
  auto test = [&](int t, const V4<T>& q, T d2, T dx, T dy, T dz) {
    if (d2 == T(0)) {
      set_error(err, POT_ERR_COINCIDENT_SITES, s);
    } else {
      T d;
      const T h = fix_zero(plane_offset(d2, ps, q.w, d), r);
      if (h <= -r) {
        empty = true;
      } else if (h < r && h - (dx * ox + dy * oy + dz * oz) / d < R) {
        if (nc < kmax) cand[row + nc] = t;
        nc++;
      }
    }
  };
  // The site's neighbour list (all sites within a reach Dv, ascending), kept
  // across the evaluations of one grid order: while the reach D stays within
  // Dv it holds every site the tests can take, so they run over it instead
  // of the grid.  Otherwise the grid walk below rebuilds it with reach
  // kVerletReach D.
  const bool use_list = vl.list != nullptr && D <= vl.reach[s];
  const bool build = vl.list != nullptr && !use_list;
  const int64_t vrow = s * (int64_t)kVerletCap;
  if (use_list) {
    const int cnt = vl.count[s];
    for (int k = 0; k < cnt && !empty; k++) {
      const int t = vl.list[vrow + k];
      const V4<T> q = sxp[t];
      T dx, dy, dz;
      const T d2 = sqdist(p, q, dx, dy, dz);
      if (d2 < D2) test(t, q, d2, dx, dy, dz);
    }
  }
  const T Dw = build ? T(kVerletReach) * D : D;  // reach of the grid walk
  const T Dw2 = Dw * Dw;
  // the rows of grid cells (fixed y and z) the walk visits
  const int cy0 = cell_coord(p.y - Dw, g.lo[1], g.inv_cs, g.dim[1]);
  const int cz0 = cell_coord(p.z - Dw, g.lo[2], g.inv_cs, g.dim[2]);
  const int nyr = cell_coord(p.y + Dw, g.lo[1], g.inv_cs, g.dim[1]) - cy0 + 1;
  const int nzr = cell_coord(p.z + Dw, g.lo[2], g.inv_cs, g.dim[2]) - cz0 + 1;
  int nv = 0;
  // One flat loop over the rows of grid cells within the reach (y, then z)
  // and their sites: the cells of a row that meet the ball of radius Dw
  // around p are one run of x, and their sites one range of grid order.
  // Each pass tests one site or opens the next row, so the lanes of a warp
  // stay on the same short path instead of diverging on nested loop
  // bounds.  Candidates come out in ascending sorted index.
  int iy = 0, iz = use_list ? nzr : 0;  // the next row to open (none with a list)
  int t = 0, b = 0;                     // the open row's sites [t, b)
  while (!empty) {
    if (t < b) {
      if (t != s) {
        const V4<T> q = sxp[t];
        T dx, dy, dz;
        const T d2 = sqdist(p, q, dx, dy, dz);
        if (d2 < Dw2) {
          if (build) {
            if (nv < kVerletCap) vl.list[vrow + nv] = t;
            nv++;
          }
          if (d2 < D2) test(t, q, d2, dx, dy, dz);
        }
      }
      t++;
      continue;
    }
    if (iz >= nzr) break;
    const int cy = cy0 + iy, cz = cz0 + iz;
    if (++iy == nyr) {
      iy = 0;
      iz++;
    }
    // distance from p to the row's cells in y and z (a cell on the grid's
    // edge extends past it: sites outside the box are in the edge cells)
    const T zlo = g.lo[2] + cz * g.cs;
    T ez = fmax(T(0), fmax(zlo - p.z, p.z - (zlo + g.cs)));
    if (cz == 0 && p.z < zlo) ez = T(0);
    if (cz == g.dim[2] - 1 && p.z > zlo) ez = T(0);
    const T ylo = g.lo[1] + cy * g.cs;
    T ey = fmax(T(0), fmax(ylo - p.y, p.y - (ylo + g.cs)));
    if (cy == 0 && p.y < ylo) ey = T(0);
    if (cy == g.dim[1] - 1 && p.y > ylo) ey = T(0);
    const T e2 = ey * ey + ez * ez;
    if (e2 >= Dw2) continue;
    // the row's cells within Dw of p: x within hw of p.x (widened by 1e-3
    // so that rounding never drops a cell the ball meets; the sites are
    // tested against Dw one by one)
    const T hw = sqrt(Dw2 - e2) * T(1.001);
    const int row = (cz * g.dim[1] + cy) * g.dim[0];
    t = cell_start[row + cell_coord(p.x - hw, g.lo[0], g.inv_cs, g.dim[0])];
    b = cell_start[row + cell_coord(p.x + hw, g.lo[0], g.inv_cs, g.dim[0]) + 1];
  }
  if (build) {
    // a walk cut short (empty cell) or a list over capacity is no list
    const bool ok = !empty && nv <= kVerletCap;
    vl.count[s] = ok ? nv : 0;
    vl.reach[s] = ok ? Dw : T(0);
  }
  const T lo = srad_lo[s];
  const bool collapsed = R - lo <= T(0.03) * R;
  // too many planes for the cell kernel's shared window, and not yet known
  // to need that many in this evaluation
  const bool soft = nw + nc > kPlaneCap && !(need[s] & kNeedBig);
  if (!empty && !(nc > kmax) && soft && collapsed) need[s] |= kNeedBig;  // a big cell from now on
  if (empty) {
    meta[s] = kMetaEmpty;
  } else if (nc > kmax || (soft && !collapsed)) {
    // over capacity, or too many planes for the window while a smaller
    // radius may still do: bisect; a cell becomes a big cell only when its
    // bracket has collapsed
    if (collapsed) {
      set_error(err, POT_ERR_NEIGHBOUR_OVERFLOW, s);
      meta[s] = kMetaEmpty;
    } else {
      srad[s] = lo > T(0) ? T(0.5) * (lo + R) : T(0.5) * R;
      meta[s] = kMetaEmpty | kMetaRetry;
    }
  } else {
    meta[s] = (nw + nc) | (wmask << kMetaWallShift);
    // more planes than the cell kernel's crossing sets hold: the big-cell kernel
    if (nw + nc > kSmallPlanes) big_list[atomicAdd(big_count, 1)] = (int32_t)s;
  }
}

// ---------------------------------------------------------------------------
// facet geometry

template <typename T>
struct alignas(2 * sizeof(T)) P2 {
  T x, y;
};

template <typename T>
struct Facet {
  T area, omega, mx, my, mz;
  T rm2;  // squared distance from the site of the facet's farthest point
  int overflow;
  int arc;  // the restricted facet has a circular edge (it reaches the sphere)
};

// Orthonormal basis (u, v) of the plane with unit normal n, branch-free:
// Duff, Burgess, Christensen, Hery, Kensler, Liani, Villemin (2017),
// "Building an Orthonormal Basis, Revisited", JCGT 6(1).
template <typename T>
__device__ __forceinline__ void onb(T nx, T ny, T nz, T& ux, T& uy, T& uz, T& vx, T& vy, T& vz) {
  T sg = copysign(T(1), nz);
  T a = T(-1) / (sg + nz);
  T b = nx * ny * a;
  ux = T(1) + sg * nx * nx * a;
  uy = sg * b;
  uz = -sg * nx;
  vx = b;
  vy = sg + ny * ny * a;
  vz = -ny;
}

template <typename T>
__device__ __forceinline__ void isect(T a1, T b1, T c1, T a2, T b2, T c2, T& x, T& y) {
  T det = a1 * b2 - a2 * b1;
  if (det == T(0)) det = T(1e-30);
  T inv = T(1) / det;
  x = (c1 * b2 - c2 * b1) * inv;
  y = (a1 * c2 - a2 * c1) * inv;
}

// Facet fi of a cell whose planes are pl[0..m): (n, h) with y.n <= h.
// A plane whose line passes clearly outside the polygon's bounding circle
// (radius^2 rp2 around the disk centre) is dismissed without visiting the
// vertices (nor clipping by a line that only grazes a vertex within
// rounding).
// Returns area, signed solid angle at the site and first moment (about the site).
// rm2 is measured from the security-ball centre p + o (oa = |o|).
template <typename T, typename IdT>
__device__ Facet<T> facet_eval(const V4<T>* __restrict__ pl, int m, int fi, T ps, T r, T ox, T oy,
                               T oz, T oa, bool want_extent) {
  Facet<T> out = {T(0), T(0), T(0), T(0), T(0), T(0), 0, 0};
  const V4<T> P = pl[fi];
  const T h = P.w;
  const T rho2 = ps - h * h;
  if (!(rho2 > T(0))) return out;
  const T rho = sqrt(rho2);
  T ux, uy, uz, vx, vy, vz;
  onb(P.x, P.y, P.z, ux, uy, uz, vx, vy, vz);
  const T B = T(2) * rho;

  // polygon: line ids (plane index, or kSq + 0..3 for the square around
  // the disk) and vertices; vertex k = intersection of lines k-1 and k
  constexpr int kSq = sizeof(IdT) == 1 ? 0xfc : 0xfffc;
  static_assert(sizeof(IdT) == 2 || kPlaneCap <= 0xfc, "plane indices must stay below the square's ids");
  static_assert(kBigPlanes <= 0xfffc, "plane indices must stay below the square's ids");
  IdT lid[2][kMaxLines];
  // vertex coordinates as (x, y) pairs: one 8-byte local access per vertex
  P2<T> pv[2][kMaxLines];
  int cur = 0, nl = 4;
  lid[0][0] = kSq; lid[0][1] = kSq + 1; lid[0][2] = kSq + 2; lid[0][3] = kSq + 3;
  pv[0][0] = P2<T>{-B, -B};
  pv[0][1] = P2<T>{B, -B};
  pv[0][2] = P2<T>{B, B};
  pv[0][3] = P2<T>{-B, B};

  auto line = [&](int id, T& a, T& b, T& c) {
    if (id >= kSq) {
      a = (id == kSq + 1) ? T(1) : ((id == kSq + 3) ? T(-1) : T(0));
      b = (id == kSq + 2) ? T(1) : ((id == kSq) ? T(-1) : T(0));
      c = B;
    } else {
      const V4<T> G = pl[id];
      a = ux * G.x + uy * G.y + uz * G.z;
      b = vx * G.x + vy * G.y + vz * G.z;
      c = G.w - h * (P.x * G.x + P.y * G.y + P.z * G.z);
    }
  };

  T rp2 = T(2) * B * B;  // squared radius of a circle around the polygon
  for (int gi = 0; gi < m; gi++) {
    if (gi == fi) continue;
    T a, b, c;
    line(gi, a, b, c);
    T len2 = a * a + b * b;
    if (len2 == T(0)) {  // parallel plane: keeps all or nothing
      if (c < T(0)) return out;
      continue;
    }
    // |c| >= rho |(a,b)|: the line misses the disk, which lies inside the
    // half-plane (c > 0) or outside it (no facet)
    const T cc = c * c;
    if (cc >= rho2 * len2) {
      if (c > T(0)) continue;
      return out;
    }
    // every vertex v has a.v <= |(a,b)| |v| < c: the polygon is inside
    if (c > T(0) && cc >= len2 * rp2 * T(1.0001)) continue;
    unsigned om = 0;
    for (int k = 0; k < nl; k++) {
      const P2<T> v = pv[cur][k];
      if (a * v.x + b * v.y > c) om |= 1u << k;
    }
    if (om == 0) continue;
    const unsigned full = (1u << nl) - 1u;
    if (om == full) return out;
    unsigned prev = ((om << 1) | (om >> (nl - 1))) & full;  // bit k: vertex k-1 outside
    int s = __ffs(om & ~prev) - 1;                          // first outside vertex of a run
    unsigned nxt = ((om >> 1) | (om << (nl - 1))) & full;   // bit k: vertex k+1 outside
    unsigned em = om & ~nxt;                                // last outside vertex of a run
    unsigned rot = s == 0 ? em : (((em >> s) | (em << (nl - s))) & full);
    int e = s + __ffs(rot) - 1;
    if (e >= nl) e -= nl;
    int cnt = s - e - 1;
    if (cnt < 0) cnt += nl;
    cnt += 1;  // lines e, e+1, ..., s-1 stay
    if (cnt + 1 > kMaxLines) {
      out.overflow = 1;
      return out;
    }
    const int nx = cur ^ 1;
    T mr2 = T(0);
    for (int k = 0; k < cnt; k++) {
      int idx = e + k;
      if (idx >= nl) idx -= nl;
      lid[nx][k] = lid[cur][idx];
      const P2<T> v = pv[cur][idx];
      const T vx = v.x, vy = v.y;
      pv[nx][k] = v;
      if (k > 0) mr2 = fmax(mr2, vx * vx + vy * vy);
    }
    lid[nx][cnt] = (IdT)gi;
    T a2, b2, c2;
    line(lid[cur][e], a2, b2, c2);
    T x0, y0;
    isect(a, b, c, a2, b2, c2, x0, y0);
    pv[nx][0] = P2<T>{x0, y0};
    int sm1 = s == 0 ? nl - 1 : s - 1;
    line(lid[cur][sm1], a2, b2, c2);
    T x1, y1;
    isect(a2, b2, c2, a, b, c, x1, y1);
    pv[nx][cnt] = P2<T>{x1, y1};
    mr2 = fmax(mr2, x0 * x0 + y0 * y0);
    rp2 = fmax(mr2, x1 * x1 + y1 * y1);
    nl = cnt + 1;
    cur = nx;
  }

  // restrict to the disk and integrate over the fan from the disk centre
  const T sg = h >= T(0) ? T(1) : T(-1);
  const T ah = fabs(h), h2 = h * h;
  const T rho3 = rho2 * rho / T(3);
  const T sect_om = sg - h / r;
  T area = T(0), omg = T(0), mx = T(0), my = T(0);
  // the security-ball centre in the facet's frame (disk centre at h n);
  // rm2 collects squared distances of the facet's extreme points from it
  const T ou = ux * ox + uy * oy + uz * oz, ov = vx * ox + vy * oy + vz * oz;
  const T on = h - (P.x * ox + P.y * oy + P.z * oz);
  const T on2 = on * on;
  const T ol = sqrt(ou * ou + ov * ov);
  const T far2 = (rho + ol) * (rho + ol) + on2;  // the circle's farthest point
  T rm2 = T(0);
  // Each polygon edge p -> q splits at its crossings x1, x2 with the circle
  // into an arc piece p -> x1 (a sector of the disk), the chord piece
  // x1 -> x2 (a triangle with the disk centre) and an arc piece x2 -> q;
  // pieces that do not occur (real == false) add exact zeros.  Every lane
  // runs all three pieces of each edge, so the lanes of a warp do not
  // diverge on which pieces their edges have.
  auto sector = [&](T ax, T ay, T bx, T by, bool real) {
    const T cr = real ? ax * by - ay * bx : T(0);
    const T dt = ax * bx + ay * by;
    const T phi = atan2(cr, dt);
    area += T(0.5) * rho2 * phi;
    omg += phi * sect_om;
    const T na = sqrt(ax * ax + ay * ay), nb = sqrt(bx * bx + by * by);
    const bool dirs = na > T(0) && nb > T(0);
    const T ina = dirs ? T(1) / na : T(0), inb = dirs ? T(1) / nb : T(0);
    if (real && dirs) {
      mx += rho3 * (by * inb - ay * ina);
      my += rho3 * (ax * ina - bx * inb);
    }
    if (!want_extent || !real) return;
    if (!dirs) {
      rm2 = fmax(rm2, far2);
      return;
    }
    // the arc from direction a to direction b: its end points, and the
    // circle's farthest point from the centre when it lies on the arc
    const T ex = rho * ax * ina - ou, ey = rho * ay * ina - ov;
    const T fx = rho * bx * inb - ou, fy = rho * by * inb - ov;
    rm2 = fmax(rm2, fmax(ex * ex + ey * ey, fx * fx + fy * fy) + on2);
    if (ol > T(0)) {
      const T gx = -ou, gy = -ov;  // direction of the farthest point
      const T c1 = ax * gy - ay * gx, c2 = gx * by - gy * bx;
      const bool half = dt < T(0) && fabs(cr) <= T(1e-6) * na * nb;
      if (half || (cr >= T(0) ? (c1 >= T(0) && c2 >= T(0)) : (c1 <= T(0) && c2 <= T(0))))
        rm2 = fmax(rm2, far2);
    }
  };
  auto tri = [&](T ax, T ay, T bx, T by, bool real) {
    const T cr = real ? ax * by - ay * bx : T(0);
    const T dt = ax * bx + ay * by;
    const T la = sqrt(ax * ax + ay * ay + h2), lb = sqrt(bx * bx + by * by + h2);
    const T den = la * lb + ah * (la + lb) + dt + h2;
    const T ta = T(0.5) * cr;
    area += ta;
    omg += sg * T(2) * atan2(cr, den);
    mx += ta * (ax + bx) * T(1.0 / 3.0);
    my += ta * (ay + by) * T(1.0 / 3.0);
  };
  bool arc = false;
  for (int k = 0; k < nl; k++) {
    int k2 = k + 1 == nl ? 0 : k + 1;
    const P2<T> vk = pv[cur][k], vq = pv[cur][k2];
    T pxk = vk.x, pyk = vk.y, qx = vq.x, qy = vq.y;
    const T pk2 = pxk * pxk + pyk * pyk;
    if (want_extent && pk2 <= rho2) {  // a polygon vertex inside the disk
      const T ex = pxk - ou, ey = pyk - ov;
      rm2 = fmax(rm2, ex * ex + ey * ey + on2);
    }
    T dx = qx - pxk, dy = qy - pyk;
    T a2 = dx * dx + dy * dy;
    if (a2 == T(0)) continue;
    T b2 = pxk * dx + pyk * dy;
    T c2 = pk2 - rho2;
    T disc = b2 * b2 - a2 * c2;
    // no crossing: the whole edge is an arc piece (t1 = t2 = 1)
    T t1 = T(1), t2 = T(1);
    if (disc > T(0)) {
      const T sq = sqrt(disc);
      t1 = fmin(fmax((-b2 - sq) / a2, T(0)), T(1));
      t2 = fmin(fmax((-b2 + sq) / a2, T(0)), T(1));
    }
    // a clamped crossing is the vertex itself, exactly
    T x1 = t1 == T(0) ? pxk : (t1 == T(1) ? qx : pxk + t1 * dx);
    T y1 = t1 == T(0) ? pyk : (t1 == T(1) ? qy : pyk + t1 * dy);
    T x2 = t2 == T(0) ? pxk : (t2 == T(1) ? qx : pxk + t2 * dx);
    T y2 = t2 == T(0) ? pyk : (t2 == T(1) ? qy : pyk + t2 * dy);
    const bool s1 = t1 > T(0), s2 = t2 < T(1);
    sector(pxk, pyk, x1, y1, s1);
    tri(x1, y1, x2, y2, t2 > t1);
    sector(x2, y2, qx, qy, s2);
    arc = arc || s1 || s2;
  }
  out.rm2 = rm2;
  out.arc = arc && area > T(0);
  out.area = area;
  out.omega = omg;
  out.mx = h * P.x * area + ux * mx + vx * my;
  out.my = h * P.y * area + uy * mx + vy * my;
  out.mz = h * P.z * area + uz * mx + vz * my;
  return out;
}

// Plane f of cell `cell` (walls first in order -x,+x,-y,+y,-z,+z, then the
// candidate bisectors in ascending sorted index).
// S is the storage type of sxp (the FP64 re-evaluation of FP32 cells widens
// the stored float values exactly).
template <typename T, typename S = T>
__device__ __forceinline__ void plane_of(int f, int64_t cell, const V4<T>& p, int mt, T r,
                                         const V4<S>* __restrict__ sxp,
                                         const int32_t* __restrict__ cand, int kmax,
                                         const Box<T>& box, V4<T>& pl, T& pd, int& pj) {
  int wmask = (mt >> kMetaWallShift) & 63;
  int nw = __popc(wmask);
  if (f < nw) {
    int w = 0, k = f;
    for (w = 0; w < 6; w++) {
      if (wmask & (1 << w)) {
        if (k == 0) break;
        k--;
      }
    }
    T h = fix_zero(wall_offset(p, w, box.lo, box.hi), r);
    int ax = w >> 1;
    T sgn = (w & 1) ? T(1) : T(-1);
    pl.x = ax == 0 ? sgn : T(0);
    pl.y = ax == 1 ? sgn : T(0);
    pl.z = ax == 2 ? sgn : T(0);
    pl.w = h;
    pd = T(0);
    pj = -1;
  } else {
    int t = cand[cell * kmax + (f - nw)];
    const V4<S> qs = sxp[t];
    const V4<T> q = {T(qs.x), T(qs.y), T(qs.z), T(qs.w)};
    T dx, dy, dz;
    T d2 = sqdist(p, q, dx, dy, dz);
    T d;
    T h = fix_zero(plane_offset(d2, p.w, q.w, d), r);
    T inv = T(1) / d;
    pl.x = dx * inv;
    pl.y = dy * inv;
    pl.z = dz * inv;
    pl.w = h;
    pd = d;
    pj = t;
  }
}

template <typename T>
struct CellAcc {
  T hA, om, nx, ny, nz, hx, hy, hz, dg, rm2;
  T wg;      // sum over wall facets of |B| / (2 h): the walls' P1 Laplacian weight
  int nfac;  // facets of positive area
  int arc;   // facets with a circular edge
};

template <typename T>
__device__ __forceinline__ void acc_facet(CellAcc<T>& a, const V4<T>& pl, T pd, int pj,
                                          const Facet<T>& fo) {
  a.hA += pl.w * fo.area;
  a.om += fo.omega;
  a.nx += pl.x * fo.area;
  a.ny += pl.y * fo.area;
  a.nz += pl.z * fo.area;
  a.hx += pl.w * fo.mx;
  a.hy += pl.w * fo.my;
  a.hz += pl.w * fo.mz;
  if (pj >= 0)
    a.dg += fo.area / (T(2) * pd);
  else
    a.wg += fo.area / (T(2) * pl.w);
  a.rm2 = fmax(a.rm2, fo.rm2);
  a.nfac += fo.area > T(0) ? 1 : 0;
  a.arc += fo.arc;
}

// The walls' part of the surface tension of a cell: over its wall facets
// (area, plane: outward normal n and the site's distance h), the sums of
// |B| n / 2 and of |B| n / (2 h), added into v[0..6).
template <typename T>
__device__ __forceinline__ void wall_vec(T area, const V4<T>& pl, T* v) {
  const T wb = area / (T(2) * pl.w);
  v[0] += T(0.5) * area * pl.x;
  v[1] += T(0.5) * area * pl.y;
  v[2] += T(0.5) * area * pl.z;
  v[3] += wb * pl.x;
  v[4] += wb * pl.y;
  v[5] += wb * pl.z;
}

// Segmented sum over lanes [lane, last] into the segment's first lane (max
// for rm2), a fixed tree: after level off, a lane holds its lanes [lane,
// min(lane + 2 off - 1, last)].  span (the same in every lane) bounds the
// segments' lengths.  All fields go level by level: the shuffles of a level
// are independent.  The levels stay a loop (the cell kernel's code size,
// see below).
template <typename T>
__device__ __forceinline__ void seg_reduce(CellAcc<T>& a, int lane, int last, int span = 32) {
#pragma unroll 1
  for (int off = 1; off < 32; off <<= 1) {
    if (off >= span) break;
    const T hA = __shfl_down_sync(kFull, a.hA, off), om = __shfl_down_sync(kFull, a.om, off);
    const T nx = __shfl_down_sync(kFull, a.nx, off), ny = __shfl_down_sync(kFull, a.ny, off);
    const T nz = __shfl_down_sync(kFull, a.nz, off), hx = __shfl_down_sync(kFull, a.hx, off);
    const T hy = __shfl_down_sync(kFull, a.hy, off), hz = __shfl_down_sync(kFull, a.hz, off);
    const T dg = __shfl_down_sync(kFull, a.dg, off), wg = __shfl_down_sync(kFull, a.wg, off);
    const T rm2 = __shfl_down_sync(kFull, a.rm2, off);
    const int nfac = __shfl_down_sync(kFull, a.nfac, off), arc = __shfl_down_sync(kFull, a.arc, off);
    if (lane + off <= last) {
      a.hA += hA;
      a.om += om;
      a.nx += nx;
      a.ny += ny;
      a.nz += nz;
      a.hx += hx;
      a.hy += hy;
      a.hz += hz;
      a.dg += dg;
      a.wg += wg;
      a.rm2 = fmax(a.rm2, rm2);
      a.nfac += nfac;
      a.arc += arc;
    }
  }
}

struct CellOut {
  void* rcell;
  const uint8_t* need;
  void* vol;
  void* karea;
  void* diag;
  void* cen;
  int32_t* row_cnt;
  double* grad;
  const double* snu;
  void* wallw;  // the walls' Laplacian weight per cell (optional)
  void* wallv;  // the walls' surface-tension vectors per cell (6 values, optional)
  int32_t* fix_count;  // FP32 kernels: ill-conditioned cells for the FP64 pass (NULL: none)
  int32_t* fix_list;
};

// An FP32 cell whose rounding can exceed the parity bounds is recomputed in
// FP64 (k_cells_fix64).  The FP32 volume carries an absolute error of a few
// ulp of the ball volume when a spherical part is present (r|K|/3 with
// |K| = psi (4 pi [inside] - sum Omega)) or when the site is outside its
// polytope (pyramids of both signs): about 2e-7 of the ball, so a cell below
// 1/20 of its ball could miss 1e-5 relative.  The Hessian diagonal carries
// r times the solid-angle rounding, about 2e-6 r: a diagonal below 0.1 r
// could miss 1e-5 relative.  Cells without a spherical part and with the
// site inside are sums of positive pyramids: well conditioned.  Where two
// lines of a facet cross inside its disk at an angle whose sine is below
// kIllSine, their vertex, computed by each of the two tasks from its own
// line, moves by the FP32 rounding over that sine, and the facets' solid
// angles no longer close up: measured against the FP64 oracle on 30k
// random balls whose radii double across the box, such cells reach 2.8e-6
// of their ball (sines near 4e-3; cells whose smallest sine is above 1.5e-2
// stay below 9e-7, 7e-6 relative where they are not recomputed), so a cell
// with such a vertex is also recomputed below a third of its ball.
constexpr float kFixBallOverVol = 20.0f;
constexpr float kFixDiagOverR = 0.1f;
constexpr float kFixIllBallOverVol = 3.0f;

// T: arithmetic of the cell, S: storage type of the outputs.  Returns true
// when an FP32 cell is ill-conditioned (see above).
template <typename T, typename S = T>
__device__ __forceinline__ bool write_cell(int64_t cell, const V4<T>& p, bool empty, bool inside,
                                           bool qout, bool full, const CellAcc<T>& a, int cnt, T oa,
                                           const CellOut& o, const T* wv) {
  const T ps = p.w;
  T V = T(0), K = T(0), dg = T(0);
  T cx = p.x, cy = p.y, cz = p.z;
  if (!empty && ps > T(0)) {
    const T r = sqrt(ps);
    // A spherical part of the boundary is bounded by circular facet edges:
    // a cell with facets none of which has an arc is a polytope inside its
    // ball (or its ball misses the polytope), |K| = 0 exactly.  The formula
    // would leave a few ulp of 4 pi psi there, a volume error that grows
    // like psi^(3/2) in deep fluid.
    if (a.nfac > 0 && (a.arc & kArcMask) == 0) {
      K = T(0);
    } else {
      K = ps * (T(4.0 * 3.14159265358979323846) * (inside ? T(1) : T(0)) - a.om);
      K = fmax(K, T(0));
    }
    V = (a.hA + r * K) * T(1.0 / 3.0);
    dg = a.dg + K / (T(2) * r);
    if (V > T(0)) {
      T iv = T(0.25) / V;
      cx += (a.hx - ps * a.nx) * iv;
      cy += (a.hy - ps * a.ny) * iv;
      cz += (a.hz - ps * a.nz) * iv;
    }
  }
  // farthest point of the cell from its security-ball centre c = p + o,
  // decided geometrically (|K| carries rounding noise of a few ulp of
  // 4 pi psi): over the facet vertices and, where facets leave their disks,
  // their circles; the spherical part's farthest point from c is on those
  // circles or is q = p - r o/|o| (distance r + |o|) when no plane cuts q
  // off; a cell without facets is the full ball (r + |o| too)
  T rc = T(0);
  if (!empty && ps > T(0)) {
    const T rq = sqrt(ps) + oa;
    if (full || a.nfac == 0)  // the whole ball (any cell inside it is within rq)
      rc = V > T(0) ? rq : T(0);
    else if ((a.arc & kArcMask) > 0 && !qout && oa > T(0))
      rc = fmax(sqrt(a.rm2), rq);
    else
      rc = sqrt(a.rm2);
  }
  ((S*)o.rcell)[cell] = (S)rc;
  ((S*)o.vol)[cell] = (S)V;
  ((S*)o.karea)[cell] = (S)K;
  ((S*)o.diag)[cell] = (S)dg;
  S* cen = (S*)o.cen;
  cen[3 * cell + 0] = (S)cx;
  cen[3 * cell + 1] = (S)cy;
  cen[3 * cell + 2] = (S)cz;
  o.row_cnt[cell] = cnt;
  if (o.grad) o.grad[cell] = o.snu[cell] - (double)(S)V;
  if (o.wallw) ((S*)o.wallw)[cell] = empty ? S(0) : (S)a.wg;
  if (o.wallv) {
    S* ov = (S*)o.wallv + 6 * cell;
    for (int k = 0; k < 6; k++) ov[k] = empty ? S(0) : (S)wv[k];
  }
  if (sizeof(T) != 4 || empty || !(ps > T(0)) || (K == T(0) && inside)) return false;
  const T r = sqrt(ps);
  const T ball = T(4.0 * 3.14159265358979323846 / 3.0) * ps * r;
  return V * T(kFixBallOverVol) < ball || dg < T(kFixDiagOverR) * r ||
         (a.arc >= kIllFlag && V * T(kFixIllBallOverVol) < ball);
}

// Append an ill-conditioned FP32 cell to the FP64 list and put its full
// plane list back into its candidate row (the cell kernel rewrote the row in
// place into its Hessian columns): j of its bisector planes, in plane order
// after the walls.  Rare (no fluid cell is listed), so kept out of line: the
// cell kernel's code stays smaller.
__device__ __noinline__ void flag_fix(int64_t cell, int m, int nw, const int* pj, int kmax,
                                         int32_t* cand, int32_t* fix_count, int32_t* fix_list) {
  fix_list[atomicAdd(fix_count, 1)] = (int32_t)cell;
  for (int f = nw; f < m; f++) cand[cell * kmax + (f - nw)] = pj[f];
}

// ---------------------------------------------------------------------------
// cell kernel (cells of at most kSmallPlanes planes)
//
// A restricted facet B_f is the disk of plane f (centre h_f n_f, radius
// rho_f = sqrt(psi - h_f^2)) cut by the half-planes that the other planes
// trace on it (Sec. 3.4).  Only the lines that cross the disk matter: a plane
// whose line misses the disk keeps all of it or none (the facet is empty).
// Whether the line of two planes f and g crosses the ball is symmetric in f
// and g -- the line's distance from the site is below r --, so it is decided
// once per pair of planes.
//
// With the crossing lines G_f, the boundary of B_f is a cycle of chord
// segments and circular arcs, and area, solid angle at the site (Sec. 3.3)
// and first moment are sums over it of fan pieces from the disk centre: a
// triangle per segment, a sector per arc.  Each crossing line g gives one
// task: its chord [-w, w] (direction with the facet on its left) clipped by
// the other lines of G_f is the segment of g on the boundary, when not empty;
// if the end of the chord survives the clipping, an arc starts there and
// runs counter-clockwise to the nearest chord start of a line of G_f (the
// first point where the circle leaves the facet).  A line whose whole chord
// lies behind the arc's start does not end it; the start of a line whose
// cut-off arc contains the arc's start (possible only where three boundary
// pieces meet, within rounding) ends it at once.  A facet crossed by no line
// is its whole disk.  No polygon is stored: every task runs in registers on
// the planes in the warp's shared window.
//
// The kernel is bound by instruction issue and, among its stalls, most by
// instruction fetch: its loops are kept rolled (#pragma unroll 1), which
// made it 20 % faster than with the compiler's unrolling.
constexpr int kWin = 96;  // plane slots of a warp's window

// Warps per block: the window of every warp lives in static shared memory,
// so the FP64 kernel runs half as many warps per block.
template <typename T>
struct CellCfg {
  static constexpr int warps = sizeof(T) == 4 ? kCellWarps : kCellWarps / 2;
};

// Per-cell accumulators of a window, in shared memory.
template <typename T>
struct CellSlot {
  CellAcc<T> a;
  int neg;      // some plane has h < 0 (the site is outside the polytope)
  int qout;     // some plane excludes the sphere point farthest from the security centre
  int emitted;  // Hessian entries written so far
};


// Monotone stand-in for the counter-clockwise angle in [0, 2 pi) between
// two directions, from their cross and dot products: 0 at the same
// direction, 2 opposite, approaching 4 just behind.
__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fast_div(double a, double b) { return a / b; }
__device__ __forceinline__ float rsqrt_t(float a) { return rsqrtf(a); }
__device__ __forceinline__ double rsqrt_t(double a) { return 1.0 / sqrt(a); }

template <typename T>
__device__ __forceinline__ T pangle(T cr, T dt) {
  const T s = fabs(cr) + fabs(dt);
  const T x = s > T(0) ? fast_div(dt, s) : T(1);
  return cr >= T(0) ? T(1) - x : T(3) + x;
}

// Line-decision tolerances of the task kernel (relative to the disk radius):
// a line whose half chord is below kTangent rho touches the disk (it cuts a
// cap of area below 1e-9 rho^2, none of the facet, or all of it); two lines
// within kCoincide (angle, and offset relative to rho) are one line.
template <typename T>
struct LineTol;
template <>
struct LineTol<float> {
  static constexpr float kTangent2 = 1e-6f;  // (1e-3)^2
  static constexpr float kCoincide = 4e-6f;
};
template <>
struct LineTol<double> {
  static constexpr double kTangent2 = 1e-14;
  static constexpr double kCoincide = 1e-12;
};

// A crossing line of a facet in the facet's frame, staged in shared memory
// by its task for the other tasks of the same facet: unit normal (a, b) and
// offset c (the facet is on the side a x + b y <= c), chord start S and end
// Q (counter-clockwise: the facet lies on the left of S -> Q), plane index
// within the cell and whether it crosses the disk by more than a touch.
template <typename T>
struct LineRec {
  T a, b, c, sx, sy, qx, qy;
  int gl;  // plane index | live << 8
};

template <typename T>
struct TaskOut {
  T area, om, mx, my, rm2;
  int arc;
};

// Frame of facet f: the disk and the security-ball centre in it.
template <typename T>
struct FacetFrame {
  T h, rho2, rho, ux, uy, uz, vx, vy, vz, sect_om, ou, ov, on2, ol, far2;
};

template <typename T>
__device__ __forceinline__ FacetFrame<T> facet_frame(const V4<T>& P, T ps, T ir, T ox, T oy, T oz) {
  FacetFrame<T> F;
  F.h = P.w;
  F.rho2 = ps - P.w * P.w;
  F.rho = F.rho2 > T(0) ? sqrt(F.rho2) : T(0);
  onb(P.x, P.y, P.z, F.ux, F.uy, F.uz, F.vx, F.vy, F.vz);
  F.sect_om = (P.w >= T(0) ? T(1) : T(-1)) - P.w * ir;
  F.ou = F.ux * ox + F.uy * oy + F.uz * oz;
  F.ov = F.vx * ox + F.vy * oy + F.vz * oz;
  const T on = P.w - (P.x * ox + P.y * oy + P.z * oz);
  F.on2 = on * on;
  F.ol = sqrt(F.ou * F.ou + F.ov * F.ov);
  F.far2 = (F.rho + F.ol) * (F.rho + F.ol) + F.on2;  // the circle's farthest point
  return F;
}

// Line of plane G in the frame of facet plane P (unit normal, offset), its
// chord and liveness.
template <typename T>
__device__ __forceinline__ LineRec<T> line_rec(const V4<T>& P, const FacetFrame<T>& F, const V4<T>& G,
                                               int g) {
  LineRec<T> L;
  const T a = F.ux * G.x + F.uy * G.y + F.uz * G.z, b = F.vx * G.x + F.vy * G.y + F.vz * G.z;
  const T c = G.w - F.h * (P.x * G.x + P.y * G.y + P.z * G.z);
  const T il = rsqrt_t(a * a + b * b);
  L.a = a * il;
  L.b = b * il;
  L.c = c * il;
  const T w2 = F.rho2 - L.c * L.c;
  const bool live = w2 > LineTol<T>::kTangent2 * F.rho2;
  const T w = live ? sqrt(w2) : T(0);
  // foot c (a, b), direction (-b, a)
  L.sx = L.c * L.a + w * L.b;
  L.sy = L.c * L.b - w * L.a;
  L.qx = L.c * L.a - w * L.b;
  L.qy = L.c * L.b + w * L.a;
  L.gl = g | (live ? 256 : 0);
  return L;
}

// The crossing point of two crossing lines of a facet (the lower plane
// index first: every task that needs it computes the same bits).
template <typename T>
__device__ __forceinline__ void meet(const LineRec<T>& L1, const LineRec<T>& L2, T& x, T& y) {
  const T det = L1.a * L2.b - L2.a * L1.b;
  const T id = T(1) / det;
  x = (L1.c * L2.b - L2.c * L1.b) * id;
  y = (L1.a * L2.c - L2.a * L1.c) * id;
}

// One task of facet f: its line `own` (rec[me]) among the facet's lines
// rec[lo..hi], or the facet's whole disk when no line crosses it (own.gl <
// 0).  Moments are in the facet frame about the disk centre; rm2 is the
// squared distance of the task's farthest boundary point from the security
// centre, when want_extent.
template <typename T>
__device__ __forceinline__ TaskOut<T> facet_task(const FacetFrame<T>& F, const LineRec<T>* rec,
                                                 int me, int lo, int hi, int lowest,
                                                 bool want_extent) {
  TaskOut<T> out = {T(0), T(0), T(0), T(0), T(0), 0};
  constexpr T kPi = T(3.14159265358979323846);
  if (!(F.rho2 > T(0))) return out;
  if (lo > hi) {  // no line crosses the disk: the whole disk
    out.area = kPi * F.rho2;
    out.om = T(2) * kPi * F.sect_om;
    out.arc = 1;
    out.rm2 = want_extent ? F.far2 : T(0);
    return out;
  }
  const LineRec<T> G = rec[me];
  const int g = G.gl & 255;
  const bool own_live = (G.gl & 256) != 0;
  // a touching line with the disk centre on its far side leaves no facet
  if (!own_live && !(G.c > T(0))) return out;
  const T Fx = G.c * G.a, Fy = G.c * G.b, dx = -G.b, dy = G.a;
  const T w2 = F.rho2 - G.c * G.c;
  const T w = own_live ? sqrt(w2) : T(0);
  T t0 = -w, t1 = w;
  int k0 = -1, k1 = -1;  // the lines that cut the chord's start and end
  bool none = !own_live, dead = false, other_live = false;
  // a line crossing g's chord inside the disk at a small angle: the vertex
  // they make moves by the rounding of e over s (FP32 cells with one are
  // recomputed in FP64 when small against their ball, see write_cell)
  bool ill = false;
  // the chord end B = Q, where an arc starts if it survives; the nearest
  // chord start ahead of it: first g's own
  const T Bx = G.qx, By = G.qy;
  T ecr = Bx * G.sy - By * G.sx, edt = Bx * G.sx + By * G.sy;
  T Ex = G.sx, Ey = G.sy;
  T best = pangle(ecr, edt);
#pragma unroll 1
  for (int j = lo; j <= hi; j++) {
    if (j == me) continue;
    const LineRec<T> K = rec[j];
    if (!(K.gl & 256)) {  // k touches the disk: all of it or none
      if (!(K.c > T(0))) dead = true;
      continue;
    }
    other_live = true;
    if (!own_live) continue;
    const T s = K.a * dx + K.b * dy;    // sin of the angle between the lines
    const T e = K.c - (K.a * Fx + K.b * Fy);  // distance of g's foot from line k
    if (fabs(s) <= LineTol<T>::kCoincide && fabs(e) <= LineTol<T>::kCoincide * F.rho) {
      // one line: the lower plane index carries it; opposite half-planes
      // leave no area
      if (K.a * G.a + K.b * G.b < T(0) || (K.gl & 255) < g) none = true;
      continue;
    }
    if (s != T(0)) {
      const T te = fast_div(e, s);
      if (s > T(0)) {
        if (te < t1) {
          t1 = te;
          k1 = j;
        }
      } else if (te > t0) {
        t0 = te;
        k0 = j;
      }
      ill = ill || (fabs(s) < T(kIllSine) && fabs(te) < w);
    } else if (e < T(0)) {
      none = true;
    }
    const T scr = Bx * K.sy - By * K.sx, sdt = Bx * K.sx + By * K.sy;
    T ps_ = pangle(scr, sdt);
    // the arc start inside k's cut-off arc (from its start to its end):
    // only within rounding, where the arc has no length
    if (pangle(Bx * K.qy - By * K.qx, Bx * K.qx + By * K.qy) < ps_) ps_ = T(0);
    if (ps_ < best) {
      best = ps_;
      ecr = scr;
      edt = sdt;
      Ex = K.sx;
      Ey = K.sy;
    }
  }
  if (dead) return out;
  if (!own_live) {
    // touching lines only: the whole disk, counted by the lowest one
    if (!other_live && g == lowest) {
      out.area = kPi * F.rho2;
      out.om = T(2) * kPi * F.sect_om;
      out.arc = 1;
      out.rm2 = want_extent ? F.far2 : T(0);
    }
    return out;
  }
  if (none || !(t0 < t1)) return out;
  // the segment of g on the boundary: triangle piece from the disk centre.
  // A clipped end is the crossing of g with the line that cuts it, computed
  // from the two lines in plane order, so that the task of that line gets
  // the same vertex to the last bit (where two lines are nearly parallel,
  // e / s moves the vertex far along them, and two tasks computing it
  // each from its own line would leave a gap or an overlap between their
  // pieces)
  T Ax = Fx + t0 * dx, Ay = Fy + t0 * dy;
  T Cx = Fx + t1 * dx, Cy = Fy + t1 * dy;
  if (k0 >= 0) meet(rec[min(me, k0)], rec[max(me, k0)], Ax, Ay);
  if (k1 >= 0) meet(rec[min(me, k1)], rec[max(me, k1)], Cx, Cy);
  {
    const T ah = fabs(F.h), h2 = F.h * F.h;
    const T cr = Ax * Cy - Ay * Cx;
    const T dt = Ax * Cx + Ay * Cy;
    const T la = sqrt(Ax * Ax + Ay * Ay + h2), lb = sqrt(Cx * Cx + Cy * Cy + h2);
    const T den = la * lb + ah * (la + lb) + dt + h2;
    const T ta = T(0.5) * cr;
    out.area = ta;
    out.om = (F.h >= T(0) ? T(2) : T(-2)) * atan2(cr, den);
    out.mx = ta * (Ax + Cx) * T(1.0 / 3.0);
    out.my = ta * (Ay + Cy) * T(1.0 / 3.0);
    if (want_extent) {
      const T ex = Ax - F.ou, ey = Ay - F.ov, fx = Cx - F.ou, fy = Cy - F.ov;
      out.rm2 = fmax(ex * ex + ey * ey, fx * fx + fy * fy) + F.on2;
    }
  }
  if (t1 == w && best > T(0)) {
    // the arc from the chord end B to E, counter-clockwise
    // (the angle from the same cross and dot products that ranked E)
    T phi = atan2(ecr, edt);
    if (phi < T(0)) phi += T(2) * kPi;
    out.area += T(0.5) * F.rho2 * phi;
    out.om += phi * F.sect_om;
    out.mx += F.rho2 * T(1.0 / 3.0) * (Ey - By);
    out.my += F.rho2 * T(1.0 / 3.0) * (Bx - Ex);
    out.arc = 1;
    // the circle's farthest point from the security centre, if on the arc
    if (want_extent && F.ol > T(0)) {
      const T gx = -F.rho * F.ou / F.ol, gy = -F.rho * F.ov / F.ol;
      if (pangle(Bx * gy - By * gx, Bx * gx + By * gy) <= best) out.rm2 = fmax(out.rm2, F.far2);
    }
  }
  if (ill) out.arc += kIllFlag;
  return out;
}

// the same segmented sums (max for rm2) over a facet's task results
template <typename T>
__device__ __forceinline__ void seg_task(TaskOut<T>& k, int lane, int last, int span) {
#pragma unroll 1
  for (int off = 1; off < 32; off <<= 1) {
    if (off >= span) break;
    const T area = __shfl_down_sync(kFull, k.area, off), om = __shfl_down_sync(kFull, k.om, off);
    const T mx = __shfl_down_sync(kFull, k.mx, off), my = __shfl_down_sync(kFull, k.my, off);
    const T rm2 = __shfl_down_sync(kFull, k.rm2, off);
    const int arc = __shfl_down_sync(kFull, k.arc, off);
    if (lane + off <= last) {
      k.area += area;
      k.om += om;
      k.mx += mx;
      k.my += my;
      k.rm2 = fmax(k.rm2, rm2);
      k.arc += arc;
    }
  }
}

// A warp's window: the planes of consecutive cells, the crossing sets, the
// task prefix and the per-facet sums of the tasks.
template <typename T>
struct Window {
  V4<T> pl[kWin];   // plane (n, h) of each slot
  T pd[kWin];       // distance to the neighbour (0 for a wall)
  int pj[kWin];     // neighbour (sorted index), -1 for a wall
  unsigned mask[kWin];  // lines crossing the slot's disk (bit = plane of the same cell)
  int tpre[kWin + 1];   // first task of each slot
  uint8_t owner[kWin];  // window cell of each slot
  uint8_t dead[kWin];   // a plane keeps none of the slot's disk
  T fa[kWin], fo[kWin], fx[kWin], fy[kWin], fr[kWin];  // facet area, solid angle, moment, extent
  uint8_t farc[kWin];
  LineRec<T> rec[32];  // the lines of the current round's tasks
  uint8_t rstart[32];  // the round's slot (from its first) starting at each task offset
  int cex[33];      // first slot of each window cell
  int cpp[33];      // first plane pair of each window cell
  CellSlot<T> sc[32];
};


// inclusive warp prefix sum
__device__ __forceinline__ int warp_incl(int v, int lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    int t = __shfl_up_sync(kFull, v, off);
    if (lane >= off) v += t;
  }
  return v;
}

// last index i in [0, n) with a[i] <= x (a ascending, a[0] <= x)
__device__ __forceinline__ int last_le(const int* a, int n, int x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a[mid] <= x)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// One warp per task of up to 32 consecutive cells (grid order), processed in
// windows: as many of its cells as have all their planes fit in the warp's
// kWin slots.  Per window: (A) one lane per slot builds a plane; (B) one
// lane per pair of planes of a cell decides whether their line crosses the
// ball (then each is in the other's crossing set) or else whether one keeps
// none of the other's disk; (C) one lane per task (facet, crossing line)
// integrates its segment and arc, and a segmented warp sum per facet is
// added, in round order, to the facet's sums in shared memory; (D) one lane
// per slot turns its facet into the cell's pyramid, moment and Hessian
// terms, writes the facet to the cell's Hessian row in plane order when its
// area counts, and a segmented warp sum per cell is added to the cell's
// accumulator; (E) one lane per cell writes it.  All sums are in a fixed
// order (deterministic).  Cells of more than kSmallPlanes planes are the
// big-cell kernel's.
template <typename T>
__global__ void __launch_bounds__(CellCfg<T>::warps * 32, sizeof(T) == 4 ? 6 : 2)
    k_cells(int64_t n, const V4<T>* __restrict__ sxp, const int32_t* __restrict__ meta,
            int32_t* cand, int kmax, Box<T> box, T* stage_vals, const T* __restrict__ soff,
            const T* __restrict__ srad, CellOut o, int32_t* chunk_next, int32_t* err) {
  constexpr int W = CellCfg<T>::warps;
  __shared__ Window<T> s_win[W];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Window<T>& S = s_win[wid];
  (void)err;
  // each warp takes the next chunk of kCellsPerWarp cells until none is
  // left: a warp that finishes early takes more, so no window waits idle
  // for a slow warp of its block
  const int64_t nchunk = (n + kCellsPerWarp - 1) / kCellsPerWarp;
  for (;;) {
    int chunk = 0;
    if (lane == 0) chunk = atomicAdd(chunk_next, 1);
    chunk = __shfl_sync(kFull, chunk, 0);
    if (chunk >= nchunk) break;
    const int64_t c0 = (int64_t)chunk * kCellsPerWarp;
    const int64_t c1 = c0 + kCellsPerWarp < n ? c0 + kCellsPerWarp : n;
    int64_t base = c0;
    while (base < c1) {
      // window: lane w stands for cell base + w
      const int64_t cell = base + lane;
      const bool valid = cell < c1;
      const bool todo = valid && o.need[cell];  // cells finished in an earlier pass take no slot
      const int mt = todo ? meta[cell] : 0;
      const int m = mt & kMetaPlanes;
      const bool mine = todo && m <= kSmallPlanes;  // larger cells are the big-cell kernel's
      const int slots = mine ? m : 0;
      const int incl = warp_incl(slots, lane);
      const int excl = incl - slots;
      // a prefix of the cells (m <= kSmallPlanes <= kWin, so the first always fits)
      const bool take = valid && incl <= kWin;
      const int ncell = __popc(__ballot_sync(kFull, take));
      const int total = __shfl_sync(kFull, incl, ncell - 1);
      const int np = take ? slots * (slots - 1) / 2 : 0;
      const int pincl = warp_incl(np, lane);
      V4<T> pw = {};
      T rw = T(0), irw = T(0), oxw = T(0), oyw = T(0), ozw = T(0);
      bool fullw = false;  // the security ball contains the site's ball: exact without an extent
      if (take && mine) {
        pw = sxp[cell];
        rw = pw.w > T(0) ? sqrt(pw.w) : T(0);
        irw = rw > T(0) ? T(1) / rw : T(0);
        oxw = soff[3 * cell + 0];
        oyw = soff[3 * cell + 1];
        ozw = soff[3 * cell + 2];
        fullw = srad[cell] >= rw + sqrt(oxw * oxw + oyw * oyw + ozw * ozw);
        S.sc[lane].a = CellAcc<T>{};
        S.sc[lane].neg = 0;
        S.sc[lane].qout = 0;
        S.sc[lane].emitted = 0;
      }
      if (lane < ncell) {
        S.cex[lane] = excl;
        S.cpp[lane] = pincl - np;
      }
      if (lane == ncell - 1) {
        S.cex[ncell] = total;
        S.cpp[ncell] = pincl;
      }
      __syncwarp();
      const int ptot = S.cpp[ncell];

      // (A) the window's planes, one slot per lane
#pragma unroll 1
      for (int t0 = 0; t0 < total; t0 += 32) {
        const int t = t0 + lane;
        const int ow = t < total ? last_le(S.cex, ncell, t) : 0;
        const int omt = __shfl_sync(kFull, mt, ow);
        const V4<T> op = {__shfl_sync(kFull, pw.x, ow), __shfl_sync(kFull, pw.y, ow),
                          __shfl_sync(kFull, pw.z, ow), __shfl_sync(kFull, pw.w, ow)};
        const T orr = __shfl_sync(kFull, rw, ow);
        if (t < total) {
          plane_of(t - S.cex[ow], base + ow, op, omt, orr, sxp, cand, kmax, box, S.pl[t], S.pd[t],
                   S.pj[t]);
          S.owner[t] = (uint8_t)ow;
          S.mask[t] = 0u;
          S.dead[t] = 0;
          S.fa[t] = T(0);
          S.fo[t] = T(0);
          S.fx[t] = T(0);
          S.fy[t] = T(0);
          S.fr[t] = T(0);
          S.farc[t] = 0;
        }
      }
      __syncwarp();

      // (B) pairs of planes of each cell: k-th pair of a cell of mc planes is
      // (f, f + s mod mc), s = k / mc + 1, f = k mod mc (each unordered pair once)
#pragma unroll 1
      for (int p0 = 0; p0 < ptot; p0 += 32) {
        const int p = p0 + lane;
        const int c = p < ptot ? last_le(S.cpp, ncell, p) : 0;
        const T psc = __shfl_sync(kFull, pw.w, c);
        if (p < ptot) {
          const int k = p - S.cpp[c];
          const int sb = S.cex[c];
          const int mc = S.cex[c + 1] - sb;
          // k / mc: k < 496 and mc <= 32 put (k + 1/2) / mc at least 1/64
          // from an integer, far beyond the error of the fast divide
          const int s = __float2int_rz(__fdividef((float)k + 0.5f, (float)mc)) + 1;
          const int f = k - (s - 1) * mc;
          int g = f + s;
          if (g >= mc) g -= mc;
          const V4<T> F = S.pl[sb + f], G = S.pl[sb + g];
          const T cxx = F.y * G.z - F.z * G.y, cyy = F.z * G.x - F.x * G.z, czz = F.x * G.y - F.y * G.x;
          const T len2 = cxx * cxx + cyy * cyy + czz * czz;  // 1 - (n_f . n_g)^2
          const T cs = F.x * G.x + F.y * G.y + F.z * G.z;
          const T cf = G.w - F.w * cs;  // g's line offset in f's plane: > 0 keeps f's disk centre
          const T cg = F.w - G.w * cs;
          bool cross = false;
          if (len2 > T(0)) {
            // the line of f and g crosses the open ball iff
            // h_f^2 - 2 cs h_f h_g + h_g^2 < psi (1 - cs^2), written as
            // (h_f -+ h_g)^2 (1 + |cs|) +- 2 len2 h_f h_g < psi len2 (1 + |cs|)
            // (upper signs for cs >= 0), without cancellation
            const T a1 = T(1) + fabs(cs);
            const T dd = cs >= T(0) ? F.w - G.w : F.w + G.w;
            const T fg = (cs >= T(0) ? T(2) : T(-2)) * len2 * F.w * G.w;
            cross = dd * dd * a1 + fg < psc * len2 * a1;
          }
          if (cross) {
            atomicOr(&S.mask[sb + f], 1u << g);
            atomicOr(&S.mask[sb + g], 1u << f);
          } else {
            const bool parallel = !(len2 > T(0));
            if (parallel ? cf < T(0) : !(cf > T(0))) S.dead[sb + f] = 1;
            if (parallel ? cg < T(0) : !(cg > T(0))) S.dead[sb + g] = 1;
          }
        }
      }
      __syncwarp();

      // (C) tasks: a live facet has one per crossing line, or one for its
      // whole disk; first the task prefix over the slots
      int carry = 0;
#pragma unroll 1
      for (int t0 = 0; t0 < total; t0 += 32) {
        const int t = t0 + lane;
        int nt = 0;
        if (t < total && !S.dead[t]) {
          const int pc = __popc(S.mask[t]);
          nt = pc > 0 ? pc : 1;
        }
        const int inc = warp_incl(nt, lane);
        if (t < total) S.tpre[t] = carry + inc - nt;
        carry += __shfl_sync(kFull, inc, 31);
      }
      if (lane == 0) S.tpre[total] = carry;
      __syncwarp();
      const int ttot = carry;
      // rounds of whole facets (a facet has at most kSmallPlanes - 1 tasks):
      // each task stages its line for the other tasks of its facet.  A
      // round looks at the 32 slots from sR: lane l's slot starts its tasks
      // at st (relative to R) and has nt of them; the slots whose tasks end
      // by 32 form a prefix (st + nt is the next slot's st) and make the
      // round; their facet starts, as bits, give each task lane its facet's
      // first and last lane, and the slot is read back by its start.
#pragma unroll 1
      for (int R = 0, sR = 0; R < ttot;) {
        const int sl = sR + lane;
        const bool sv = sl < total;
        const int st = sv ? S.tpre[sl] - R : 64;
        const int nt = sv ? S.tpre[sl + 1] - R - st : 0;
        const bool fits = sv && st + nt <= 32;
        const int span = __reduce_max_sync(kFull, fits ? st + nt : 0);
        const unsigned starts = __reduce_or_sync(kFull, fits && nt > 0 ? 1u << st : 0u);
        if (fits && nt > 0) S.rstart[st] = (uint8_t)lane;
        const int sR0 = sR;
        sR += __popc(__ballot_sync(kFull, fits));
        __syncwarp();
        const int Rend = R + span;
        const bool act = lane < span;
        const unsigned upto = 0xffffffffu >> (31 - lane);  // bits 0..lane
        const int fs = act ? 31 - __clz(starts & upto) : lane;
        const unsigned above = starts & ~upto;
        const int slot = act ? sR0 + S.rstart[fs] : 0;
        const int c = act ? S.owner[slot] : 0;
        const T psc = __shfl_sync(kFull, pw.w, c);
        const T oir = __shfl_sync(kFull, irw, c);
        const T sox = __shfl_sync(kFull, oxw, c), soy = __shfl_sync(kFull, oyw, c),
                soz = __shfl_sync(kFull, ozw, c);
        const bool ofull = __shfl_sync(kFull, fullw, c);
        const int head = fs;
        const int last = !act ? lane : above ? __ffs(above) - 2 : span - 1;
        FacetFrame<T> fr = {};
        unsigned M = 0u;
        if (act) {
          const int sb = S.cex[c];
          const V4<T> P = S.pl[slot];
          fr = facet_frame(P, psc, oir, sox, soy, soz);
          M = S.mask[slot];
          if (M) {
            const int g = (int)__fns(M, 0, lane - head + 1);
            S.rec[lane] = line_rec(P, fr, S.pl[sb + g], g);
          }
        }
        __syncwarp();
        TaskOut<T> tk = {T(0), T(0), T(0), T(0), T(0), 0};
        if (act)
          tk = M ? facet_task(fr, S.rec, lane, head, last, __ffs(M) - 1, !ofull)
                 : facet_task(fr, S.rec, lane, 1, 0, 0, !ofull);
        seg_task(tk, lane, last, __reduce_max_sync(kFull, last - head + 1));
        if (act && lane == head) {
          S.fa[slot] = tk.area;
          S.fo[slot] = tk.om;
          S.fx[slot] = tk.mx;
          S.fy[slot] = tk.my;
          S.fr[slot] = tk.rm2;
          S.farc[slot] = (uint8_t)(((tk.arc & kArcMask) > 0 ? 1 : 0) | (tk.arc >= kIllFlag ? 2 : 0));
        }
        __syncwarp();
        R = Rend;
      }

      // (D) facets: pyramid, moment and Hessian terms per slot, emission, and
      // a segmented sum per cell
#pragma unroll 1
      for (int t0 = 0; t0 < total; t0 += 32) {
        const int t = t0 + lane;
        const bool inr = t < total;
        const int ow = inr ? S.owner[t] : 0;
        const T ops = __shfl_sync(kFull, pw.w, ow);
        const T orr = __shfl_sync(kFull, rw, ow);
        const T sox = __shfl_sync(kFull, oxw, ow), soy = __shfl_sync(kFull, oyw, ow),
                soz = __shfl_sync(kFull, ozw, ow);
        CellAcc<T> a = {};
        bool neg = false, qo = false, emit = false;
        T area = T(0);
        if (inr) {
          const V4<T> P = S.pl[t];
          area = S.fa[t];
          Facet<T> fo = {};
          fo.area = area;
          fo.omega = S.fo[t];
          fo.rm2 = S.fr[t];
          fo.arc = ((S.farc[t] & 1) && area > T(0) ? 1 : 0) + ((S.farc[t] & 2) ? kIllFlag : 0);
          T ux, uy, uz, vx, vy, vz;
          onb(P.x, P.y, P.z, ux, uy, uz, vx, vy, vz);
          const T mx = S.fx[t], my = S.fy[t];
          fo.mx = P.w * P.x * area + ux * mx + vx * my;
          fo.my = P.w * P.y * area + uy * mx + vy * my;
          fo.mz = P.w * P.z * area + uz * mx + vz * my;
          acc_facet(a, P, S.pd[t], S.pj[t], fo);
          neg = P.w < T(0);
          // the sphere point farthest from the security centre, q = p - r o/|o|,
          // is cut off by this plane (clearly: n . (q - p) > h + 1e-6 r)
          const T soa = sqrt(sox * sox + soy * soy + soz * soz);
          qo = soa > T(0) && -orr * (P.x * sox + P.y * soy + P.z * soz) > (P.w + T(1e-6) * orr) * soa;
          emit = S.pj[t] >= 0 && area > Real<T>::kEmitArea * ops;
        }
        const int cs0 = S.cex[ow];
        const int lo = inr ? max(cs0 - t0, 0) : lane;
        const int hi = inr ? min(S.cex[ow + 1] - 1 - t0, 31) : lane;
        seg_reduce(a, lane, hi, __reduce_max_sync(kFull, hi - lo + 1));
        const unsigned segmask = inr ? ((0xffffffffu >> (31 - hi)) & ~((1u << lo) - 1u)) : 0u;
        const unsigned negm = __ballot_sync(kFull, neg);
        const unsigned qm = __ballot_sync(kFull, qo);
        const unsigned emm = __ballot_sync(kFull, emit);
        const int done = inr ? S.sc[ow].emitted : 0;
        if (emit) {
          const int rank = done + __popc(emm & segmask & ((1u << lane) - 1u));
          const int64_t at = (base + ow) * kmax + rank;
          cand[at] = S.pj[t];
          stage_vals[at] = -area / (T(2) * S.pd[t]);
        }
        __syncwarp();
        if (inr && lane == lo) {
          CellAcc<T>& sa = S.sc[ow].a;
          sa.hA += a.hA;
          sa.om += a.om;
          sa.nx += a.nx;
          sa.ny += a.ny;
          sa.nz += a.nz;
          sa.hx += a.hx;
          sa.hy += a.hy;
          sa.hz += a.hz;
          sa.dg += a.dg;
          sa.wg += a.wg;
          sa.rm2 = fmax(sa.rm2, a.rm2);
          sa.nfac += a.nfac;
          sa.arc += a.arc;
          S.sc[ow].neg |= (negm & segmask) != 0u;
          S.sc[ow].qout |= (qm & segmask) != 0u;
          S.sc[ow].emitted = done + __popc(emm & segmask);
        }
        __syncwarp();
      }

      // (E) the window's cells
      if (take && mine) {
        const int nw = __popc((mt >> kMetaWallShift) & 63);
        T wv[6] = {};
        if (o.wallv && !(mt & kMetaEmpty))  // the wall facets are the cell's first planes
          for (int f = 0; f < nw && f < m; f++) wall_vec(S.fa[excl + f], S.pl[excl + f], wv);
        const bool fix =
            write_cell(cell, pw, (mt & kMetaEmpty) != 0, S.sc[lane].neg == 0,
                       S.sc[lane].qout != 0 && !fullw, fullw, S.sc[lane].a, S.sc[lane].emitted,
                       sqrt(oxw * oxw + oyw * oyw + ozw * ozw), o, wv);
        if (fix && o.fix_list)
          flag_fix(cell, m, nw, S.pj + excl, kmax, cand, o.fix_count, o.fix_list);
      }
      __syncwarp();
      base += ncell;
    }
  }
}

// Cells with more planes than the cell kernel takes (kSmallPlanes): one warp per
// cell, its planes staged in the warp's slice of a global scratch (L1/L2
// resident), facets in rounds of 32 lanes with per-lane accumulators, one
// warp reduction at the end.  Line ids of the facet polygons are 16-bit.
// A fixed grid walks the list the candidate pass built (its length on the
// device), so no host round trip is needed.
template <typename T>
__global__ void __launch_bounds__(128)
    k_cells_big(const V4<T>* __restrict__ sxp, const int32_t* __restrict__ meta, int32_t* cand,
                int kmax, Box<T> box, T* stage_vals, const T* __restrict__ soff,
                const T* __restrict__ srad, const int32_t* __restrict__ big_count,
                const int32_t* __restrict__ big_list, V4<T>* big_pl, T* big_d, int* big_j,
                CellOut o, int32_t* err) {
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  V4<T>* pl = big_pl + (int64_t)gw * kBigPlanes;
  T* pd = big_d + (int64_t)gw * kBigPlanes;
  int* pj = big_j + (int64_t)gw * kBigPlanes;
  const int count = *big_count;
  for (int b = gw; b < count; b += nw) {
    const int64_t cell = big_list[b];
    const int mt = meta[cell];
    const int m = mt & kMetaPlanes;
    const V4<T> p = sxp[cell];
    const T r = p.w > T(0) ? sqrt(p.w) : T(0);
    const T ox = soff[3 * cell + 0], oy = soff[3 * cell + 1], oz = soff[3 * cell + 2];
    const T oa = sqrt(ox * ox + oy * oy + oz * oz);
    const bool full = srad[cell] >= r + oa;
    for (int f = lane; f < m; f += 32)
      plane_of(f, cell, p, mt, r, sxp, cand, kmax, box, pl[f], pd[f], pj[f]);
    __syncwarp();
    CellAcc<T> a = {};
    bool neg = false, qout = false;
    int emitted = 0;
    T warea = T(0);  // lanes 0..5 of the first round: the wall facets' areas
    for (int f0 = 0; f0 < m; f0 += 32) {
      const int f = f0 + lane;
      const bool has = f < m;
      Facet<T> fo = {};
      if (has) {
        fo = facet_eval<T, uint16_t>(pl, m, f, p.w, r, ox, oy, oz, oa, !full);
        if (f0 == 0) warea = fo.area;
        if (fo.overflow) set_error(err, POT_ERR_POLYGON_OVERFLOW, cell);
        acc_facet(a, pl[f], pd[f], pj[f], fo);
        neg |= pl[f].w < T(0);
        qout |= oa > T(0) && -r * (pl[f].x * ox + pl[f].y * oy + pl[f].z * oz) > (pl[f].w + T(1e-6) * r) * oa;
      }
      const bool emit = has && pj[f] >= 0 && fo.area > Real<T>::kEmitArea * p.w;
      const unsigned em = __ballot_sync(kFull, emit);
      if (emit) {
        const int64_t at = cell * kmax + emitted + __popc(em & ((1u << lane) - 1u));
        cand[at] = pj[f];
        stage_vals[at] = -fo.area / (T(2) * pd[f]);
      }
      emitted += __popc(em);
    }
    seg_reduce(a, lane, 31);
    const bool anyneg = __any_sync(kFull, neg);
    const bool anyq = __any_sync(kFull, qout);
    const int nw = __popc((mt >> kMetaWallShift) & 63);
    T wv[6] = {};
    for (int k = 0; k < 6; k++) {
      const T ak = __shfl_sync(kFull, warea, k);
      if (k < nw) wall_vec(ak, pl[k], wv);
    }
    if (lane == 0) {
      const bool fix = write_cell(cell, p, (mt & kMetaEmpty) != 0, !anyneg, anyq && !full, full, a,
                                  emitted, oa, o, wv);
      if (fix && o.fix_list && m <= kPlaneCap)
        flag_fix(cell, m, nw, pj, kmax, cand, o.fix_count, o.fix_list);
    }
    __syncwarp();
  }
}

// FP64 re-evaluation of the FP32 cells that write_cell found ill-conditioned
// (list built by the cell kernels of the same pass, their candidate rows
// restored): one warp per cell, the planes rebuilt in FP64 from the stored
// float sites (widened exactly, as the FP64 oracle reads them) into the
// warp's shared window, the facets in rounds of 32 lanes, and the cell's
// outputs and Hessian row rewritten (stored as float).  The emission
// threshold and the security-ball decisions stay those of the FP32 pass.
constexpr int kFixWarps = 4;

__global__ void __launch_bounds__(kFixWarps * 32)
    k_cells_fix64(const V4<float>* __restrict__ sxp, const int32_t* __restrict__ meta,
                  int32_t* cand, int kmax, Box<double> box, float* stage_vals,
                  const float* __restrict__ soff, const float* __restrict__ srad, CellOut o,
                  int32_t* err) {
  __shared__ V4<double> s_pl[kFixWarps][kPlaneCap];
  __shared__ double s_d[kFixWarps][kPlaneCap];
  __shared__ int s_j[kFixWarps][kPlaneCap];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  V4<double>* pl = s_pl[wid];
  double* pd = s_d[wid];
  int* pj = s_j[wid];
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  const int count = *o.fix_count;
  for (int b = gw; b < count; b += nwarps) {
    const int64_t cell = o.fix_list[b];
    const int mt = meta[cell];
    const int m = mt & kMetaPlanes;
    const V4<float> ps = sxp[cell];
    const V4<double> p = {ps.x, ps.y, ps.z, ps.w};
    const double r = p.w > 0.0 ? sqrt(p.w) : 0.0;
    const float oxf = soff[3 * cell + 0], oyf = soff[3 * cell + 1], ozf = soff[3 * cell + 2];
    // the security-ball decision exactly as the FP32 pass took it
    const float rf = ps.w > 0.f ? sqrtf(ps.w) : 0.f;
    const bool full = srad[cell] >= rf + sqrtf(oxf * oxf + oyf * oyf + ozf * ozf);
    const double ox = oxf, oy = oyf, oz = ozf;
    const double oa = sqrt(ox * ox + oy * oy + oz * oz);
    for (int f = lane; f < m; f += 32)
      plane_of<double, float>(f, cell, p, mt, r, sxp, cand, kmax, box, pl[f], pd[f], pj[f]);
    __syncwarp();
    CellAcc<double> a = {};
    bool neg = false, qout = false;
    int emitted = 0;
    double warea = 0.0;  // lanes 0..5 of the first round: the wall facets' areas
    for (int f0 = 0; f0 < m; f0 += 32) {
      const int f = f0 + lane;
      const bool has = f < m;
      Facet<double> fo = {};
      if (has) {
        fo = facet_eval<double, uint8_t>(pl, m, f, p.w, r, ox, oy, oz, oa, !full);
        if (f0 == 0) warea = fo.area;
        if (fo.overflow) set_error(err, POT_ERR_POLYGON_OVERFLOW, cell);
        acc_facet(a, pl[f], pd[f], pj[f], fo);
        neg |= pl[f].w < 0.0;
        qout |= oa > 0.0 && -r * (pl[f].x * ox + pl[f].y * oy + pl[f].z * oz) > (pl[f].w + 1e-6 * r) * oa;
      }
      const bool emit = has && pj[f] >= 0 && fo.area > (double)Real<float>::kEmitArea * p.w;
      const unsigned em = __ballot_sync(kFull, emit);
      if (emit) {
        const int64_t at = cell * kmax + emitted + __popc(em & ((1u << lane) - 1u));
        cand[at] = pj[f];
        stage_vals[at] = (float)(-fo.area / (2.0 * pd[f]));
      }
      emitted += __popc(em);
    }
    seg_reduce(a, lane, 31);
    const bool anyneg = __any_sync(kFull, neg);
    const bool anyq = __any_sync(kFull, qout);
    const int nw = __popc((mt >> kMetaWallShift) & 63);
    double wv[6] = {};
    for (int k = 0; k < 6; k++) {
      const double ak = __shfl_sync(kFull, warea, k);
      if (k < nw) wall_vec(ak, pl[k], wv);
    }
    if (lane == 0)
      write_cell<double, float>(cell, p, (mt & kMetaEmpty) != 0, !anyneg, anyq && !full, full, a,
                                emitted, oa, o, wv);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// security-radius passes

// largest weight of the sites of each grid cell (very negative when empty)
template <typename T>
__global__ void k_gmax(int64_t ncell, const int32_t* __restrict__ cell_start,
                       const V4<T>* __restrict__ sxp, T* gmax) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  T m = T(-1e30);
  for (int t = cell_start[c]; t < cell_start[c + 1]; t++) m = fmax(m, sxp[t].w);
  gmax[c] = m;
}

// Largest weight (clamped at 0) of the sites of each coarse cell, added by
// every lane of a warp (ok: the lane has a site): lanes that share a coarse
// cell (consecutive in grid order, so most do) combine before one atomic.
// Non-negative floating-point values order like their bit patterns as
// unsigned integers.
template <typename T>
__device__ __forceinline__ void coarse_max_add(bool ok, const V4<T>& p, const GridParams<T>& g,
                                               const Coarse<T>& co, T* cmax) {
  const int64_t key = ok ? coarse_key(p, g, co) : -1;
  const T v = ok && p.w > T(0) ? p.w : T(0);
  if constexpr (sizeof(T) == 4) {
    const unsigned grp = __match_any_sync(kFull, (unsigned long long)key);
    const unsigned m = __reduce_max_sync(grp, __float_as_uint(v));
    if (ok && (int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicMax((unsigned*)cmax + key, m);
  } else {
    if (ok)
      atomicMax((unsigned long long*)cmax + key, (unsigned long long)__double_as_longlong(v));
  }
}

// Largest of cmax over each coarse cell's 3 x 3 x 3 neighbourhood.
template <typename T>
__global__ void k_cnb(Coarse<T> co, const T* __restrict__ cmax, T* nb) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nxy = (int64_t)co.dim[0] * co.dim[1];
  if (c >= nxy * co.dim[2]) return;
  const int cx = (int)(c % co.dim[0]), cy = (int)((c / co.dim[0]) % co.dim[1]), cz = (int)(c / nxy);
  T m = T(0);
  for (int z = max(cz - 1, 0); z <= min(cz + 1, co.dim[2] - 1); z++)
    for (int y = max(cy - 1, 0); y <= min(cy + 1, co.dim[1] - 1); y++)
      for (int x = max(cx - 1, 0); x <= min(cx + 1, co.dim[0] - 1); x++)
        m = fmax(m, cmax[z * nxy + (int64_t)y * co.dim[0] + x]);
  nb[c] = m;
}

// First security ball of an evaluation.  Centre: kept from the previous
// evaluation in the same grid order (the Newton solve keeps it fixed), else
// the hint of the previous solve on these sites (centroid - site, caller
// order), else the site.  Radius: 1.25 x the cell's extent from that centre
// in the previous evaluation or at the last accepted Newton iterate,
// whichever is smaller (a rejected line-search trial can have far larger
// cells), else 1.25 x the hinted extent, else 1.5 nu^(1/3); capped at
// r + |o|, where the ball contains the site's ball.
template <typename T>
__global__ void k_srad_init(int64_t n, const V4<T>* __restrict__ sxp, const double* __restrict__ snu,
                            const T* __restrict__ rcell, int have_prev,
                            const T* __restrict__ rcell_acc, int have_acc,
                            const int32_t* __restrict__ perm, const T* __restrict__ hint,
                            int use_hint, T* srad, T* srad_lo, T* soff, uint8_t* need,
                            GridParams<T> g, Coarse<T> co, T* cmax) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const V4<T> p = s < n ? sxp[s] : V4<T>{T(0), T(0), T(0), T(0)};
  // the coarse cells' largest weights (every lane of the warp takes part)
  if (cmax) coarse_max_add(s < n, p, g, co, cmax);
  if (s >= n) return;
  const T ps = p.w;
  const T r = ps > T(0) ? sqrt(ps) : T(0);
  T ox = T(0), oy = T(0), oz = T(0);
  T prev = T(0);
  if (have_prev) {
    ox = soff[3 * s + 0];
    oy = soff[3 * s + 1];
    oz = soff[3 * s + 2];
    prev = rcell[s];
    if (have_acc && rcell_acc[s] > T(0)) prev = prev > T(0) ? fmin(prev, rcell_acc[s]) : rcell_acc[s];
  } else if (use_hint) {
    const int64_t i = perm[s];
    ox = hint[4 * i + 0];
    oy = hint[4 * i + 1];
    oz = hint[4 * i + 2];
    prev = hint[4 * i + 3];
    // a centre outside the site's ball is stale
    if (!(ox * ox + oy * oy + oz * oz < ps)) {
      ox = oy = oz = T(0);
      prev = T(0);
    }
  }
  soff[3 * s + 0] = ox;
  soff[3 * s + 1] = oy;
  soff[3 * s + 2] = oz;
  T R = r;
  if (prev > T(0))
    R = T(1.25) * prev;
  else if (snu[s] > 0.0)
    R = T(1.5) * (T)cbrt(snu[s]);
  srad[s] = fmin(R, r + sqrt(ox * ox + oy * oy + oz * oz));
  srad_lo[s] = T(0);
  need[s] = 1;
}

// After a pass: a cell inside its security ball is final.  Otherwise R is
// too small (it becomes R_lo), and the cell just built (from a subset of the
// planes) contains the true cell, so its farthest point rcell bounds the
// radius that suffices: R grows to 1.05 rcell (the margin covers the rounding
// of rcell), by a factor between 1.25 and 2, and the next pass normally
// builds a cell inside that ball.
template <typename T>
__global__ void k_need_update(int64_t n, const V4<T>* __restrict__ sxp, const T* __restrict__ rcell,
                              const int32_t* __restrict__ meta, const T* __restrict__ soff, T* srad,
                              T* srad_lo, uint8_t* need, int32_t* count) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n || !need[s]) return;
  if (meta[s] & kMetaRetry) {  // radius already reduced by the candidate pass
    atomicAdd(count, 1);
    return;
  }
  const T ps = sxp[s].w;
  const T ox = soff[3 * s + 0], oy = soff[3 * s + 1], oz = soff[3 * s + 2];
  const T rmax = (ps > T(0) ? sqrt(ps) : T(0)) + sqrt(ox * ox + oy * oy + oz * oz);
  const T R = srad[s];
  const T rc = rcell[s];
  const bool done = !(ps > T(0)) || R >= rmax || rc < R * T(1.0 - 1e-5);
  if (done) {
    need[s] = 0;
  } else {
    srad_lo[s] = R;
    srad[s] = fmin(rmax, fmin(T(2) * R, fmax(T(1.25) * R, T(1.05) * rc)));
    atomicAdd(count, 1);
  }
}

// A start with empty cells cannot enter Algorithm 1 (its KMT bound needs
// min V > 0).  For an empty cell i, psi_i <- max_j (psi_j - d_ij^2) + 0.25 d*^2
// (d* the distance to the maximising site): then h_ij > 0 for every j, so p_i
// lies strictly inside its own cell, which is no longer empty, while each
// neighbour keeps h_ji = (2 d^2 - 0.25 d*^2)/(2d) > 0 with respect to i.  Sites
// with psi_j - d^2 > psi_i lie within sqrt(psi_max - psi_i); grid cells are
// skipped when gmax - delta^2 <= psi_i.
template <typename T>
__global__ void __launch_bounds__(256)
    k_repair(int64_t n, V4<T>* sxp, T* psi_base, const T* __restrict__ vol,
             const int32_t* __restrict__ cell_start, GridParams<T> g, const T* __restrict__ gmax,
             const double* __restrict__ snu, T* psi_max, int32_t* count) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n || vol[s] > T(0)) return;
  const V4<T> p = sxp[s];
  const T ps = p.w;
  const T D = sqrt(fmax(*psi_max - ps, T(0)));
  T best = T(-1e30), bd2 = T(0);
  if (D > T(0)) {
    int c0[3], c1[3];
    const T pc[3] = {p.x, p.y, p.z};
    for (int k = 0; k < 3; k++) {
      c0[k] = cell_coord(pc[k] - D, g.lo[k], g.inv_cs, g.dim[k]);
      c1[k] = cell_coord(pc[k] + D, g.lo[k], g.inv_cs, g.dim[k]);
    }
    for (int cz = c0[2]; cz <= c1[2]; cz++)
      for (int cy = c0[1]; cy <= c1[1]; cy++)
        for (int cx = c0[0]; cx <= c1[0]; cx++) {
          const T lo3[3] = {g.lo[0] + cx * g.cs, g.lo[1] + cy * g.cs, g.lo[2] + cz * g.cs};
          T dl2 = T(0);
          for (int k = 0; k < 3; k++) {
            const T e = fmax(T(0), fmax(lo3[k] - pc[k], pc[k] - (lo3[k] + g.cs)));
            dl2 += e * e;
          }
          const int key = (cz * g.dim[1] + cy) * g.dim[0] + cx;
          if (gmax[key] - dl2 <= ps) continue;
          for (int t = cell_start[key]; t < cell_start[key + 1]; t++) {
            if (t == s) continue;
            const V4<T> q = sxp[t];
            const T dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
            const T d2 = dx * dx + dy * dy + dz * dz;
            const T v = q.w - d2;
            if (v > best) {
              best = v;
              bd2 = d2;
            }
          }
        }
  }
  T nv = ps;
  if (best > T(-1e29) && bd2 > T(0)) nv = fmax(nv, best + T(0.25) * bd2);
  // a non-positive weight is an empty ball: give it half the radius of its target
  const T floor = snu[s] > 0.0 ? T(0.25) * (T)cbrt(snu[s] * snu[s]) : T(0);
  nv = fmax(nv, floor);
  if (nv > ps) {
    sxp[s].w = nv;
    psi_base[s] = nv;
    atomicAdd(count, 1);
    if (sizeof(T) == 4)
      atomicMax((int*)psi_max, __float_as_int((float)nv));
    else
      atomicMax((unsigned long long*)psi_max, (unsigned long long)__double_as_longlong((double)nv));
  }
}

// ---------------------------------------------------------------------------
// reductions, CSR, scatter

// Per-thread terms of the residual: exact in FP64 for an FP64 evaluation;
// for an FP32 one, g = nu - V as hi + lo floats (nu split into two floats,
// the difference by an error-free two-difference) and sum g^2 in
// double-float, so that no FP64 arithmetic runs per cell.
template <typename T>
struct ResidAcc {
  double emax = 0.0, ss = 0.0, vmin = 1e300;
  int64_t nemp = 0, npl = 0;
  int mpl = 0;
  __device__ __forceinline__ void add(T v, double nu) {
    const double g = nu - (double)v;
    if (nu > 0.0) emax = fmax(emax, fabs(g) / nu);
    ss += g * g;
    vmin = fmin(vmin, (double)v);
    nemp += v <= T(0) ? 1 : 0;
  }
  __device__ __forceinline__ double sum_sq() const { return ss; }
  __device__ __forceinline__ double vol_min() const { return vmin; }
};
template <>
struct ResidAcc<float> {
  float emax = 0.f, vmin = 3.0e38f;
  DF ss;
  int64_t nemp = 0, npl = 0;
  int mpl = 0;
  __device__ __forceinline__ void add(float v, double nu) {
    const float hi = (float)nu, lo = (float)(nu - (double)hi);
    const float s = hi - v, bb = s - hi;
    const float gl = ((hi - (s - bb)) - (v + bb)) + lo;  // g = s + gl
    if (hi > 0.f) emax = fmaxf(emax, fabsf(s + gl) / hi);
    df_add_prod(ss, s, s);
    ss.lo += 2.f * s * gl;
    vmin = fminf(vmin, v);
    nemp += v <= 0.f ? 1 : 0;
  }
  __device__ __forceinline__ double sum_sq() const { return df_value(ss); }
  __device__ __forceinline__ double vol_min() const { return vmin < 3.0e38f ? vmin : 1e300; }
};

template <typename T>
__global__ void k_resid(int64_t n, const T* __restrict__ vol, const double* __restrict__ snu,
                        const int32_t* __restrict__ meta, double* part) {
  ResidAcc<T> acc;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // four cells per step with their loads issued together, added in the
  // same order as one at a time
#pragma unroll 1
  for (; i + 3 * stride < n; i += 4 * stride) {
    T v[4];
    double nu[4];
    int m[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      v[u] = vol[i + u * stride];
      nu[u] = snu[i + u * stride];
      m[u] = meta[i + u * stride] & kMetaPlanes;
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
      acc.add(v[u], nu[u]);
      acc.npl += m[u];
      acc.mpl = max(acc.mpl, m[u]);
    }
  }
  for (; i < n; i += stride) {
    acc.add(vol[i], snu[i]);
    const int m = meta[i] & kMetaPlanes;
    acc.npl += m;
    acc.mpl = max(acc.mpl, m);
  }
  double emax = acc.emax, ss = acc.sum_sq(), vmin = acc.vol_min();
  double nemp = (double)acc.nemp, npl = (double)acc.npl, mpl = (double)acc.mpl;
  __shared__ double sh[6][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int off = 16; off > 0; off >>= 1) {
    emax = fmax(emax, __shfl_down_sync(kFull, emax, off));
    ss += __shfl_down_sync(kFull, ss, off);
    vmin = fmin(vmin, __shfl_down_sync(kFull, vmin, off));
    nemp += __shfl_down_sync(kFull, nemp, off);
    npl += __shfl_down_sync(kFull, npl, off);
    mpl = fmax(mpl, __shfl_down_sync(kFull, mpl, off));
  }
  if (lane == 0) {
    sh[0][wid] = emax; sh[1][wid] = ss; sh[2][wid] = vmin;
    sh[3][wid] = nemp; sh[4][wid] = npl; sh[5][wid] = mpl;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int w = 1; w < nw; w++) {
      sh[0][0] = fmax(sh[0][0], sh[0][w]);
      sh[1][0] += sh[1][w];
      sh[2][0] = fmin(sh[2][0], sh[2][w]);
      sh[3][0] += sh[3][w];
      sh[4][0] += sh[4][w];
      sh[5][0] = fmax(sh[5][0], sh[5][w]);
    }
    for (int k = 0; k < 6; k++) part[blockIdx.x * 6 + k] = sh[k][0];
  }
}

// The block partials of k_resid over one warp: lane l takes blocks l, l + 32,
// ... in order, then a fixed shuffle tree (deterministic).
__global__ void k_resid_final(const double* __restrict__ part, int nb, double* out) {
  const int lane = threadIdx.x;
  double r[6] = {0.0, 0.0, 1e300, 0.0, 0.0, 0.0};
  for (int b = lane; b < nb; b += 32) {
    r[0] = fmax(r[0], part[6 * b + 0]);
    r[1] += part[6 * b + 1];
    r[2] = fmin(r[2], part[6 * b + 2]);
    r[3] += part[6 * b + 3];
    r[4] += part[6 * b + 4];
    r[5] = fmax(r[5], part[6 * b + 5]);
  }
  for (int off = 16; off > 0; off >>= 1) {
    r[0] = fmax(r[0], __shfl_down_sync(kFull, r[0], off));
    r[1] += __shfl_down_sync(kFull, r[1], off);
    r[2] = fmin(r[2], __shfl_down_sync(kFull, r[2], off));
    r[3] += __shfl_down_sync(kFull, r[3], off);
    r[4] += __shfl_down_sync(kFull, r[4], off);
    r[5] = fmax(r[5], __shfl_down_sync(kFull, r[5], off));
  }
  if (lane == 0)
    for (int k = 0; k < 6; k++) out[k] = r[k];
}

template <typename T>
__global__ void k_csr_copy(int64_t n, const int32_t* __restrict__ row_ptr,
                           const int32_t* __restrict__ cand, const T* __restrict__ stage, int kmax,
                           int32_t* cols, T* vals) {
  // 4 threads per row, each with up to three entries' loads in flight
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t s = t >> 2;
  int sub = (int)(t & 3);
  if (s >= n) return;
  const int a = row_ptr[s], cnt = row_ptr[s + 1] - a;
  const int32_t* cr = cand + s * kmax;
  const T* vr = stage + s * kmax;
#pragma unroll 1
  for (int k = sub; k < cnt; k += 12) {
    int c[3];
    T v[3];
#pragma unroll
    for (int u = 0; u < 3; u++) {
      if (k + 4 * u < cnt) {
        c[u] = cr[k + 4 * u];
        v[u] = vr[k + 4 * u];
      }
    }
#pragma unroll
    for (int u = 0; u < 3; u++) {
      if (k + 4 * u < cnt) {
        cols[a + k + 4 * u] = c[u];
        vals[a + k + 4 * u] = v[u];
      }
    }
  }
}

__global__ void k_user_count(int64_t n, const int32_t* __restrict__ iperm,
                             const int32_t* __restrict__ row_cnt, int32_t* ucnt) {
  int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  ucnt[o] = row_cnt[iperm[o]] + 1;
}

template <typename T>
__global__ void k_user_rows(int64_t n, const int32_t* __restrict__ iperm,
                            const int32_t* __restrict__ perm, const int32_t* __restrict__ row_ptr,
                            const int32_t* __restrict__ cand, const T* __restrict__ stage,
                            const T* __restrict__ diag, int kmax, int32_t* cols, T* vals) {
  int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const int64_t s = iperm[o];
  const int a = row_ptr[o];
  const int cnt = row_ptr[o + 1] - a;
  cols[a] = (int32_t)o;
  vals[a] = diag[s];
  for (int k = 1; k < cnt; k++) {
    int c = perm[cand[s * kmax + (k - 1)]];
    T v = stage[s * kmax + (k - 1)];
    int j = a + k - 1;
    while (j >= a && cols[j] > c) {  // insertion into the sorted prefix
      cols[j + 1] = cols[j];
      vals[j + 1] = vals[j];
      j--;
    }
    cols[j + 1] = c;
    vals[j + 1] = v;
  }
}

template <typename T>
__global__ void k_unsort(int64_t n, const int32_t* __restrict__ perm, const T* __restrict__ vol,
                         const double* __restrict__ grad, const T* __restrict__ cen,
                         const T* __restrict__ karea, const V4<T>* __restrict__ sxp, T* o_vol,
                         double* o_grad, T* o_cen, T* o_karea, T* o_psi) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  int64_t o = perm[s];
  if (o_vol) o_vol[o] = vol[s];
  if (o_grad) o_grad[o] = grad[s];
  if (o_karea) o_karea[o] = karea[s];
  if (o_cen) {
    o_cen[3 * o + 0] = cen[3 * s + 0];
    o_cen[3 * o + 1] = cen[3 * s + 1];
    o_cen[3 * o + 2] = cen[3 * s + 2];
  }
  if (o_psi) o_psi[o] = sxp[s].w;
}

template <typename T>
__global__ void k_psi_update(int64_t n, const T* __restrict__ base, const T* __restrict__ u,
                             T alpha, V4<T>* sxp, T* psi_max) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  T v = T(0);
  if (s < n) {
    v = base[s] + alpha * u[s];
    sxp[s].w = v;
  }
  block_max_to(v > T(0) ? v : T(0), psi_max);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side

template <typename T>
int cells_eval(pot_ctx* ctx, cudaStream_t st, int64_t n, const pot_domain* dom, bool want_grad,
               bool tail_resid) {
  ctx->tail_ready = false;
  Work<T>& w = ctx->work<T>();
  if (!w.grid_valid) return POT_ERR_INVALID_ARG;
  Box<T> box;
  for (int k = 0; k < 3; k++) {
    box.lo[k] = (T)dom->lo[k];
    box.hi[k] = (T)dom->hi[k];
  }
  // largest weights near each site: coarse cells of f x f x f grid cells,
  // f at least 4 and such that the neighbourhood reaches past
  // 2 sqrt(psi_max) at the grid build's weights (the largest reach of a
  // candidate); only where the workspace holds them
  Coarse<T> co = {nullptr, 1, {1, 1, 1}};
  int64_t ncc = 0;
  if (w.cmax && w.cnb) {
    int f = std::max(4, (int)ceil(2.0 * sqrt(fmax(w.grid_pmax, 0.0)) / (double)w.grid.cs + 0.5));
    for (;; f++) {
      ncc = 1;
      for (int k = 0; k < 3; k++) {
        co.dim[k] = (w.grid.dim[k] + f - 1) / f;
        ncc *= co.dim[k];
      }
      if (ncc <= w.ccap) break;
    }
    co.f = f;
    POT_CUDA(cudaMemsetAsync(w.cmax, 0, sizeof(T) * ncc, st));
  }
  note_launch();
  k_srad_init<T><<<blocks_for(n, 256), 256, 0, st>>>(
      n, w.sxp, ctx->snu, w.rcell, w.have_rcell ? 1 : 0, w.rcell_acc, w.have_acc ? 1 : 0, ctx->perm,
      w.hint, (w.use_hint && w.hint && w.hint_n == n) ? 1 : 0, w.srad, w.srad_lo, w.soff, ctx->need,
      w.grid, co, ncc > 0 ? w.cmax : nullptr);
  if (ncc > 0) {
    note_launch();
    k_cnb<T><<<blocks_for(ncc, 256), 256, 0, st>>>(co, w.cmax, w.cnb);
    co.nb = w.cnb;
  }
  CellOut o;
  o.rcell = w.rcell;
  o.need = ctx->need;
  o.vol = w.vol;
  o.karea = w.karea;
  o.wallw = w.wallw;
  o.wallv = w.wallv;
  o.diag = w.diag;
  o.cen = w.cen;
  o.row_cnt = ctx->row_cnt;
  o.grad = want_grad ? ctx->grad : nullptr;
  o.snu = ctx->snu;
  // FP32: ill-conditioned cells are listed for the FP64 re-evaluation
  const bool fix64 = sizeof(T) == 4 && ctx->fix_list != nullptr;
  o.fix_count = fix64 ? ctx->need_count + 2 : nullptr;
  o.fix_list = fix64 ? ctx->fix_list : nullptr;
  Box<double> box64;
  for (int k = 0; k < 3; k++) {
    box64.lo[k] = dom->lo[k];
    box64.hi[k] = dom->hi[k];
  }
  // neighbour lists: kept across the evaluations of one grid order when the
  // caller asked for them (a Newton solve), invalidated by the grid build
  VerletList<T> vl = {nullptr, nullptr, nullptr};
  if (w.verlet && w.vlist) vl = {w.vlist, w.vcount, w.vreach};
  // resident blocks of the cell kernel (its warps loop over chunks)
  const int64_t warps = (n + kCellsPerWarp - 1) / kCellsPerWarp;
  static const int per_sm = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_cells<T>, CellCfg<T>::warps * 32, 0) !=
        cudaSuccess)
      b = 1;
    return b;
  }();
  const int blocks = (int)std::min<int64_t>(
      (warps + CellCfg<T>::warps - 1) / CellCfg<T>::warps,
      (int64_t)std::max(per_sm, 1) * ctx->sm_count);
  int32_t* hcount = (int32_t*)(ctx->h_pinned + 24);
  ctx->last_passes = 0;
  int64_t todo = n;  // cells rebuilt in this pass
  for (int pass = 0; pass < kMaxPasses; pass++) {
    ctx->last_passes = pass + 1;
    // big cells, FP64 cells listed, the cell kernel's next chunk
    POT_CUDA(cudaMemsetAsync(ctx->need_count + 1, 0, 3 * sizeof(int32_t), st));
    note_launch();
    k_candidates<T><<<blocks_for(n, 256), 256, 0, st>>>(
        n, w.sxp, ctx->cell_start, w.grid, box, w.psi_max, w.srad, w.srad_lo, w.soff,
        ctx->need, ctx->k_max, ctx->cand, ctx->meta, ctx->need_count + 1, ctx->big_list, ctx->err,
        vl, co);
    note_launch();
    // the no-alloc entry point's context has no events: no timing there
    const bool timed = ctx->ev[6] && ctx->ev[7];
    if (timed) POT_CUDA(cudaEventRecord(ctx->ev[6], st));
    k_cells<T><<<blocks, CellCfg<T>::warps * 32, 0, st>>>(n, w.sxp, ctx->meta, ctx->cand,
                                                           ctx->k_max, box, w.stage_vals, w.soff,
                                                           w.srad, o, ctx->need_count + 3,
                                                           ctx->err);
    if (w.big_warps > 0) {
      note_launch();
      k_cells_big<T><<<w.big_warps / 4, 128, 0, st>>>(
          w.sxp, ctx->meta, ctx->cand, ctx->k_max, box, w.stage_vals, w.soff, w.srad,
          ctx->need_count + 1, ctx->big_list, w.big_pl, w.big_d, w.big_j, o, ctx->err);
    }
    if (fix64) {
      // a fixed grid walks the list (its length stays on the device)
      note_launch();
      k_cells_fix64<<<ctx->sm_count * 3, kFixWarps * 32, 0, st>>>(
          (const V4<float>*)w.sxp, ctx->meta, ctx->cand, ctx->k_max, box64, (float*)w.stage_vals,
          (const float*)w.soff, (const float*)w.srad, o, ctx->err);
    }
    if (timed) POT_CUDA(cudaEventRecord(ctx->ev[7], st));
    POT_CUDA(cudaMemsetAsync(ctx->need_count, 0, sizeof(int32_t), st));
    note_launch();
    k_need_update<T><<<blocks_for(n, 256), 256, 0, st>>>(n, w.sxp, w.rcell, ctx->meta, w.soff,
                                                          w.srad, w.srad_lo, ctx->need,
                                                          ctx->need_count);
    if (tail_resid) {
      // needed only if this is the last pass; a later pass enqueues them again
      POT_CHECK(residuals<T>(ctx, st, n, nullptr));
      POT_CUDA(cudaMemcpyAsync(ctx->h_pinned + 8, ctx->err, 2 * sizeof(int32_t),
                               cudaMemcpyDeviceToHost, st));
    }
    POT_CUDA(cudaMemcpyAsync(hcount, ctx->need_count, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    POT_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f;
    if (timed && cudaEventElapsedTime(&ms, ctx->ev[6], ctx->ev[7]) == cudaSuccess) {
      ctx->kc_launches++;
      ctx->kc_cells += todo;
      ctx->kc_ms += ms;
    }
    todo = *hcount;
    if (*hcount == 0) break;
  }
  POT_CUDA(cudaGetLastError());
  w.have_rcell = true;
  ctx->tail_ready = tail_resid;
  // cells still unresolved after the last pass are not exact
  if (*hcount != 0) return POT_ERR_NEIGHBOUR_OVERFLOW;
  return POT_OK;
}

template <typename T>
int repair_empty(pot_ctx* ctx, cudaStream_t st, int64_t n, int* repaired) {
  Work<T>& w = ctx->work<T>();
  // the largest weight of each grid cell (only the repair uses it)
  const int64_t ncell = (int64_t)w.grid.dim[0] * w.grid.dim[1] * w.grid.dim[2];
  note_launch();
  k_gmax<T><<<blocks_for(ncell, 256), 256, 0, st>>>(ncell, ctx->cell_start, w.sxp, w.gmax);
  POT_CUDA(cudaMemsetAsync(ctx->need_count, 0, sizeof(int32_t), st));
  note_launch();
  k_repair<T><<<blocks_for(n, 256), 256, 0, st>>>(n, w.sxp, w.psi_base, w.vol, ctx->cell_start, w.grid,
                                                   w.gmax, ctx->snu, w.psi_max, ctx->need_count);
  int32_t* h = (int32_t*)(ctx->h_pinned + 24);
  POT_CUDA(cudaMemcpyAsync(h, ctx->need_count, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  POT_CUDA(cudaStreamSynchronize(st));
  *repaired = h[0];
  return POT_OK;
}

template <typename T>
int residuals(pot_ctx* ctx, cudaStream_t st, int64_t n, double out[6]) {
  Work<T>& w = ctx->work<T>();
  note_launch();
  k_resid<T><<<kRedBlocks, 256, 0, st>>>(n, w.vol, ctx->snu, ctx->meta, ctx->red);
  note_launch();
  k_resid_final<<<1, 32, 0, st>>>(ctx->red, kRedBlocks, ctx->red_out);
  POT_CUDA(cudaMemcpyAsync(ctx->h_pinned, ctx->red_out, 6 * sizeof(double),
                           cudaMemcpyDeviceToHost, st));
  if (!out) return POT_OK;  // the caller's next wait on the stream completes the copy
  POT_CUDA(cudaStreamSynchronize(st));
  for (int k = 0; k < 6; k++) out[k] = ctx->h_pinned[k];
  return POT_OK;
}

int read_status(pot_ctx* ctx, cudaStream_t st, int64_t* site) {
  int32_t* h = (int32_t*)(ctx->h_pinned + 8);
  POT_CUDA(cudaMemcpyAsync(h, ctx->err, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  POT_CUDA(cudaStreamSynchronize(st));
  return status_on_host(ctx, site);
}

int status_on_host(pot_ctx* ctx, int64_t* site) {
  const int32_t* h = (const int32_t*)(ctx->h_pinned + 8);
  int code = h[0];
  int32_t s = h[1];
  if (site) *site = -1;
  if (code != 0) {
    int32_t reset[2] = {0, 0x7fffffff};
    POT_CUDA(cudaMemcpy(ctx->err, reset, sizeof(reset), cudaMemcpyHostToDevice));
    if (site && s >= 0 && s < ctx->n_max) {
      int32_t o = -1;
      POT_CUDA(cudaMemcpy(&o, ctx->perm + s, sizeof(int32_t), cudaMemcpyDeviceToHost));
      *site = o;
    }
  }
  return code;
}

template <typename T>
int csr_compact(pot_ctx* ctx, cudaStream_t st, int64_t n, int64_t* nnz_off) {
  Work<T>& w = ctx->work<T>();
  POT_CHECK(scan_exclusive(ctx, st, ctx->row_cnt, ctx->row_ptr, n));
  note_launch();
  k_csr_copy<T><<<blocks_for(n * 4, 256), 256, 0, st>>>(n, ctx->row_ptr, ctx->cand, w.stage_vals,
                                                         ctx->k_max, ctx->csr_cols, w.csr_vals);
  int32_t* h = (int32_t*)(ctx->h_pinned + 28);
  POT_CUDA(cudaMemcpyAsync(h, ctx->row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (!nnz_off) return POT_OK;  // read later with csr_nnz, after a wait on the stream
  POT_CUDA(cudaStreamSynchronize(st));
  *nnz_off = h[0];
  return POT_OK;
}

int64_t csr_nnz(const pot_ctx* ctx) { return *(const int32_t*)(ctx->h_pinned + 28); }

template <typename T>
int csr_user(pot_ctx* ctx, cudaStream_t st, int64_t n, int32_t* row_ptr, int32_t* cols, T* vals,
             int64_t cap, int64_t* nnz) {
  Work<T>& w = ctx->work<T>();
  note_launch();
  k_user_count<<<blocks_for(n, 256), 256, 0, st>>>(n, ctx->iperm, ctx->row_cnt, ctx->ucnt);
  POT_CHECK(scan_exclusive(ctx, st, ctx->ucnt, row_ptr, n));
  int32_t* h = (int32_t*)(ctx->h_pinned + 8);
  POT_CUDA(cudaMemcpyAsync(h, row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  POT_CUDA(cudaStreamSynchronize(st));
  *nnz = h[0];
  if (*nnz > cap) return POT_ERR_CAPACITY;
  note_launch();
  k_user_rows<T><<<blocks_for(n, 128), 128, 0, st>>>(n, ctx->iperm, ctx->perm, row_ptr, ctx->cand,
                                                      w.stage_vals, w.diag, ctx->k_max, cols, vals);
  POT_CUDA(cudaGetLastError());
  return POT_OK;
}

template <typename T>
int unsort_outputs(pot_ctx* ctx, cudaStream_t st, int64_t n, T* vol, double* grad, T* cen,
                   T* karea, T* psi) {
  Work<T>& w = ctx->work<T>();
  note_launch();
  k_unsort<T><<<blocks_for(n, 256), 256, 0, st>>>(n, ctx->perm, w.vol, ctx->grad, w.cen, w.karea,
                                                   w.sxp, vol, grad, cen, karea, psi);
  POT_CUDA(cudaGetLastError());
  return POT_OK;
}

template <typename T>
int psi_update(pot_ctx* ctx, cudaStream_t st, int64_t n, double alpha) {
  Work<T>& w = ctx->work<T>();
  POT_CUDA(cudaMemsetAsync(w.psi_max, 0, sizeof(T), st));
  note_launch();
  k_psi_update<T><<<blocks_for(n, 256), 256, 0, st>>>(n, w.psi_base, w.u, (T)alpha, w.sxp,
                                                       w.psi_max);
  POT_CUDA(cudaGetLastError());
  return POT_OK;
}

// hint for the next solve on these sites: centroid - site, and the cell's
// extent from the centroid (<= extent from the security centre + the
// distance between the two centres), in caller order
template <typename T>
__global__ void k_store_hint(int64_t n, const int32_t* __restrict__ perm, const V4<T>* __restrict__ sxp,
                             const T* __restrict__ cen, const T* __restrict__ soff,
                             const T* __restrict__ rcell, T* hint) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const V4<T> p = sxp[s];
  const T cx = cen[3 * s + 0] - p.x, cy = cen[3 * s + 1] - p.y, cz = cen[3 * s + 2] - p.z;
  const T dx = cx - soff[3 * s + 0], dy = cy - soff[3 * s + 1], dz = cz - soff[3 * s + 2];
  const int64_t i = perm[s];
  hint[4 * i + 0] = cx;
  hint[4 * i + 1] = cy;
  hint[4 * i + 2] = cz;
  hint[4 * i + 3] = rcell[s] > T(0) ? rcell[s] + sqrt(dx * dx + dy * dy + dz * dz) : T(0);
}

template <typename T>
int store_hint(pot_ctx* ctx, cudaStream_t st, int64_t n) {
  Work<T>& w = ctx->work<T>();
  if (!w.hint || !w.have_rcell) return POT_OK;
  note_launch();
  k_store_hint<T><<<blocks_for(n, 256), 256, 0, st>>>(n, ctx->perm, w.sxp, w.cen, w.soff, w.rcell,
                                                       w.hint);
  POT_CUDA(cudaGetLastError());
  w.hint_n = n;
  return POT_OK;
}

__global__ void k_diag(int64_t n, const int32_t* __restrict__ perm, const float* __restrict__ soff,
                       const float* __restrict__ srad, const float* __restrict__ rcell,
                       const int32_t* __restrict__ meta, float* off, float* rad, float* ext,
                       int32_t* planes) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int64_t i = perm[s];
  if (off) {
    off[3 * i + 0] = soff[3 * s + 0];
    off[3 * i + 1] = soff[3 * s + 1];
    off[3 * i + 2] = soff[3 * s + 2];
  }
  if (rad) rad[i] = srad[s];
  if (ext) ext[i] = rcell[s];
  if (planes) planes[i] = (meta[s] & kMetaEmpty) ? 0 : (meta[s] & kMetaPlanes);
}

int cell_diagnostics(pot_ctx* ctx, cudaStream_t st, int64_t n, float* off, float* rad, float* ext,
                     int32_t* planes) {
  Work<float>& w = ctx->wf;
  if (!w.sxp || !w.grid_valid || !w.have_rcell || n <= 0 || n > ctx->n_max) return POT_ERR_INVALID_ARG;
  note_launch();
  k_diag<<<blocks_for(n, 256), 256, 0, st>>>(n, ctx->perm, w.soff, w.srad, w.rcell, ctx->meta, off,
                                              rad, ext, planes);
  POT_CUDA(cudaGetLastError());
  POT_CUDA(cudaStreamSynchronize(st));
  return POT_OK;
}

#define POT_INST(T)                                                                              \
  template int cells_eval<T>(pot_ctx*, cudaStream_t, int64_t, const pot_domain*, bool, bool);    \
  template int residuals<T>(pot_ctx*, cudaStream_t, int64_t, double*);                          \
  template int repair_empty<T>(pot_ctx*, cudaStream_t, int64_t, int*);                          \
  template int csr_compact<T>(pot_ctx*, cudaStream_t, int64_t, int64_t*);                       \
  template int csr_user<T>(pot_ctx*, cudaStream_t, int64_t, int32_t*, int32_t*, T*, int64_t,    \
                           int64_t*);                                                           \
  template int unsort_outputs<T>(pot_ctx*, cudaStream_t, int64_t, T*, double*, T*, T*, T*);     \
  template int psi_update<T>(pot_ctx*, cudaStream_t, int64_t, double);                          \
  template int store_hint<T>(pot_ctx*, cudaStream_t, int64_t);
POT_INST(float)
POT_INST(double)

}  // namespace pot
