// First hit of camera rays on the fluid (Sec. 6, finding the first cell):
// depth and normal per pixel into device buffers (no window, no graphics API).
//
// The fluid, the union of the generalized Laguerre cells of Eq. 1, is the
// union of the balls B(p_i, sqrt(psi_i)) inside the box: a point of any ball
// lies in the cell of the site of least power distance, which is inside that
// site's own ball.  The first point of a ray inside it lies on the sphere of
// a cell with a free surface (|K| > 0), so with the free-surface areas the
// other balls are skipped, as the paper's impostors skip them.
//
// One thread per pixel walks the sites' grid along its ray (3D DDA from the
// box entry) and tests the balls of the sites within L cells of each cell it
// enters, L = ceil(r_max / cell size): a ball hit at t has its centre within
// L cells of the cell holding the ray point at t, so once a cell is entered
// beyond the best hit no later ball can be nearer and the walk stops.
#include <math.h>

#include "pot_internal.cuh"

namespace pot {
namespace {

struct Ray {
  float o[3], f[3], r[3], u[3];
  float th, tv;
  int w, h;
};

__device__ __forceinline__ int rcell(float x, float lo, float inv, int dim) {
  float c = (x - lo) * inv;
  int i = c < 0.f ? 0 : (int)c;
  return i >= dim ? dim - 1 : i;
}

// The interval [a, b] of the ray o + t d (|d| = 1) inside ball p; false when
// the ray misses it.  r^2 minus the squared distance from the centre to the
// ray, without cancellation between |e|^2 and b^2.
__device__ __forceinline__ bool ball_interval(const V4<float>& p, const float* o, const float* d,
                                              float& a, float& b) {
  const float ex = p.x - o[0], ey = p.y - o[1], ez = p.z - o[2];
  const float bb = ex * d[0] + ey * d[1] + ez * d[2];
  const float hx = ex - bb * d[0], hy = ey - bb * d[1], hz = ez - bb * d[2];
  const float disc = p.w - (hx * hx + hy * hy + hz * hz);
  if (!(disc >= 0.f)) return false;
  const float sq = sqrtf(disc);
  a = bb - sq;
  b = bb + sq;
  return true;
}

// The first point of the ray at or after t_from (and before t_end) inside a
// ball: the smallest max(a, t_from) over the balls whose interval [a, b]
// reaches past it.  One thread walks the sites' grid along the ray (3D DDA
// from the point at t_from) and tests the balls of the sites within
// `layers` cells of each cell it enters (layers = ceil(r_max / cell size)):
// a ball entered at t has its centre within that many cells of the cell
// holding the ray point at t, so once a cell is entered beyond the best
// entry no later ball can be nearer and the walk stops.  Balls for which
// skip(s) holds are left out.  With grow > 0 the balls' radii are grown by
// it (layers must then cover r_max + grow).  Returns the entry t (INFINITY:
// none) and the site in *hit (-1: none).
template <typename Skip>
__device__ float next_entry(const float* o, const float* d, float t_from, float t_end,
                            const V4<float>* __restrict__ sxp, const int32_t* __restrict__ cell_start,
                            const GridParams<float>& g, int layers, Skip skip, int* hit,
                            float grow = 0.f) {
  float best = INFINITY;
  int besti = -1;
  if (t_from < t_end) {
    int c[3], step[3];
    float tmax[3], tdel[3];
    for (int k = 0; k < 3; k++) {
      const float x = o[k] + t_from * d[k];
      c[k] = rcell(x, g.lo[k], g.inv_cs, g.dim[k]);
      step[k] = d[k] > 0.f ? 1 : -1;
      const float edge = g.lo[k] + (c[k] + (d[k] > 0.f ? 1 : 0)) * g.cs;
      tmax[k] = d[k] != 0.f ? (edge - o[k]) / d[k] : INFINITY;
      tdel[k] = d[k] != 0.f ? g.cs / fabsf(d[k]) : INFINITY;
    }
    float tcell = t_from;
    while (tcell <= t_end && tcell <= best) {
      const int z0 = max(c[2] - layers, 0), z1 = min(c[2] + layers, g.dim[2] - 1);
      const int y0 = max(c[1] - layers, 0), y1 = min(c[1] + layers, g.dim[1] - 1);
      const int x0 = max(c[0] - layers, 0), x1 = min(c[0] + layers, g.dim[0] - 1);
      for (int z = z0; z <= z1; z++)
        for (int y = y0; y <= y1; y++) {
          const int key0 = (z * g.dim[1] + y) * g.dim[0];
          const int a = cell_start[key0 + x0], b = cell_start[key0 + x1 + 1];
          for (int s = a; s < b; s++) {
            V4<float> p = sxp[s];
            if (!(p.w > 0.f) || skip(s)) continue;
            if (grow > 0.f) {
              const float rg = sqrtf(p.w) + grow;
              p.w = rg * rg;
            }
            float ta, tb;
            if (!ball_interval(p, o, d, ta, tb)) continue;
            const float t = fmaxf(ta, t_from);
            if (t < fminf(tb, t_end) && t < best) {
              best = t;
              besti = s;
            }
          }
        }
      // next cell along the ray
      int k = tmax[0] < tmax[1] ? (tmax[0] < tmax[2] ? 0 : 2) : (tmax[1] < tmax[2] ? 1 : 2);
      c[k] += step[k];
      if (c[k] < 0 || c[k] >= g.dim[k]) break;
      tcell = tmax[k];
      tmax[k] += tdel[k];
    }
  }
  *hit = besti;
  return best;
}

// The site of least power distance |x - p|^2 - psi at x (the generalized
// Laguerre cell holding x, Eq. 1), over the sites within `layers` grid
// cells: a site whose ball holds x is that near.  -1 when no ball holds x.
__device__ int locate(const float* x, const V4<float>* __restrict__ sxp,
                      const int32_t* __restrict__ cell_start, const GridParams<float>& g,
                      int layers) {
  int c[3];
  for (int k = 0; k < 3; k++) c[k] = rcell(x[k], g.lo[k], g.inv_cs, g.dim[k]);
  float best = 0.f;
  int besti = -1;
  for (int z = max(c[2] - layers, 0); z <= min(c[2] + layers, g.dim[2] - 1); z++)
    for (int y = max(c[1] - layers, 0); y <= min(c[1] + layers, g.dim[1] - 1); y++) {
      const int key0 = (z * g.dim[1] + y) * g.dim[0];
      const int a = cell_start[key0 + max(c[0] - layers, 0)];
      const int b = cell_start[key0 + min(c[0] + layers, g.dim[0] - 1) + 1];
      for (int s = a; s < b; s++) {
        const V4<float> p = sxp[s];
        if (!(p.w > 0.f)) continue;
        const float dx = x[0] - p.x, dy = x[1] - p.y, dz = x[2] - p.z;
        const float pw = dx * dx + dy * dy + dz * dz - p.w;
        if (besti < 0 ? pw <= 0.f : pw < best) {
          best = pw;
          besti = s;
        }
      }
    }
  return besti;
}

// camera ray of pixel (px, py): unit direction into d
__device__ __forceinline__ void pixel_ray(const Ray& cam, int px, int py, float* d) {
  const float sx = ((px + 0.5f) / cam.w * 2.f - 1.f) * cam.th;
  const float sy = (1.f - (py + 0.5f) / cam.h * 2.f) * cam.tv;
  for (int k = 0; k < 3; k++) d[k] = cam.f[k] + sx * cam.r[k] + sy * cam.u[k];
  const float il = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int k = 0; k < 3; k++) d[k] *= il;
}

// the box along the ray: [t0, t1] (t0 >= 0)
__device__ __forceinline__ void box_span(const Box<float>& box, const float* o, const float* d,
                                         float& t0, float& t1) {
  t0 = 0.f;
  t1 = INFINITY;
  for (int k = 0; k < 3; k++) {
    const float a = (box.lo[k] - o[k]) / d[k], b = (box.hi[k] - o[k]) / d[k];
    t0 = fmaxf(t0, fminf(a, b));
    t1 = fminf(t1, fmaxf(a, b));
  }
}

__global__ void __launch_bounds__(256)
    k_render(Ray cam, Box<float> box, const V4<float>* __restrict__ sxp,
             const int32_t* __restrict__ perm, const float* __restrict__ karea,
             const int32_t* __restrict__ cell_start, GridParams<float> g, int layers,
             float* depth, float* normal) {
  const int px = blockIdx.x * blockDim.x + threadIdx.x;
  const int py = blockIdx.y * blockDim.y + threadIdx.y;
  if (px >= cam.w || py >= cam.h) return;
  float d[3];
  pixel_ray(cam, px, py, d);
  float t0, t1;
  box_span(box, cam.o, d, t0, t1);
  int besti = -1;
  const float best = next_entry(
      cam.o, d, t0, t1, sxp, cell_start, g, layers,
      [&](int s) { return karea && !(karea[perm[s]] > 0.f); }, &besti);
  const int pix = py * cam.w + px;
  depth[pix] = besti >= 0 ? best : -1.f;
  if (normal) {
    float nx = 0.f, ny = 0.f, nz = 0.f;
    if (besti >= 0) {
      const V4<float> p = sxp[besti];
      const float ir = rsqrtf(p.w);
      nx = (cam.o[0] + best * d[0] - p.x) * ir;
      ny = (cam.o[1] + best * d[1] - p.y) * ir;
      nz = (cam.o[2] + best * d[2] - p.z) * ir;
    }
    normal[3 * pix + 0] = nx;
    normal[3 * pix + 1] = ny;
    normal[3 * pix + 2] = nz;
  }
}

// Volume traversal (Sec. 6): one thread per ray walks the fluid cell by
// cell.  Inside cell c the ray leaves at the nearest of: the far point of
// c's sphere (into air), the box, or the radical plane of a restricted-facet
// neighbour j of c (the Hessian row's columns: the planes that bound the
// cell inside its ball), crossed towards j (then the walk goes on in j).
// The cell is the intersection of its ball, the box and those half-spaces,
// convex, so the nearest crossing is its exit.  In air, the next entry into
// the fluid is the next ball entry along the ray (the grid walk above, from
// just past the exit), and the cell entered is located by power distance;
// this replaces the walk through the unrestricted diagram.  A crossing the
// cell-by-cell walk misses (a facet below the emission threshold, rounding
// at an edge) only leaves the fluid early, and the air search re-enters it
// at once.  Outputs per pixel: first entry t (-1: none), length inside the
// fluid, last exit t (-1), cells visited.  kMaxVisits bounds the walk.
constexpr int kMaxVisits = 1 << 15;

__global__ void __launch_bounds__(128)
    k_render_volume(Ray cam, Box<float> box, const V4<float>* __restrict__ sxp,
                    const float* __restrict__ karea, const int32_t* __restrict__ cell_start,
                    GridParams<float> g, int layers, const int32_t* __restrict__ row_ptr,
                    const int32_t* __restrict__ cols, float* first, float* thick, float* last,
                    int32_t* visits) {
  const int px = blockIdx.x * blockDim.x + threadIdx.x;
  const int py = blockIdx.y * blockDim.y + threadIdx.y;
  if (px >= cam.w || py >= cam.h) return;
  float d[3];
  pixel_ray(cam, px, py, d);
  float t0, t1;
  box_span(box, cam.o, d, t0, t1);
  float tf = -1.f, tl = -1.f, len = 0.f;
  int nv = 0;
  float t = t0;
  while (t < t1 && nv < kMaxVisits) {
    const float t_round = t;
    // next entry into the fluid (balls of cells without free surface
    // cannot be entered from air)
    int s = -1;
    const float te = next_entry(
        cam.o, d, t, t1, sxp, cell_start, g, layers,
        [&](int q) { return !(karea[q] > 0.f); }, &s);
    if (s < 0) break;
    t = te;
    const float x[3] = {cam.o[0] + t * d[0], cam.o[1] + t * d[1], cam.o[2] + t * d[2]};
    int c = locate(x, sxp, cell_start, g, layers);
    if (c < 0) c = s;
    if (tf < 0.f) tf = t;
    // the walk through the fluid
    while (nv < kMaxVisits) {
      nv++;
      const V4<float> p = sxp[c];
      float ta, tb;
      float tn = t1;
      if (ball_interval(p, cam.o, d, ta, tb))
        tn = fminf(tn, tb);
      else
        tn = t;  // grazing: leave at once
      int next = -1;
      const float ox = cam.o[0] - p.x, oy = cam.o[1] - p.y, oz = cam.o[2] - p.z;
      for (int k = row_ptr[c]; k < row_ptr[c + 1]; k++) {
        const int j = cols[k];
        const V4<float> q = sxp[j];
        // radical plane: (y - p) . m = (|m|^2 + psi_c - psi_j) / 2, m = p_j - p_c
        const float mx = q.x - p.x, my = q.y - p.y, mz = q.z - p.z;
        const float md = mx * d[0] + my * d[1] + mz * d[2];
        if (!(md > 0.f)) continue;  // not towards j
        const float hm = 0.5f * (mx * mx + my * my + mz * mz + p.w - q.w);
        const float tj = (hm - (ox * mx + oy * my + oz * mz)) / md;
        if (tj > t && tj < tn) {
          tn = tj;
          next = j;
        }
      }
      if (tn > t) len += tn - t;
      t = fmaxf(t, tn);
      if (next < 0) break;
      c = next;
    }
    tl = t;
    if (t >= t1) break;
    // a step past the exit point into air: a few ulp of t at least (a step
    // below t's resolution would leave t where it is), and a round that
    // made no progress steps on as well
    const float step = fmaxf(1e-6f * g.cs, 4.8e-7f * fabsf(t));
    t = fmaxf(t, t_round) + step;
  }
  const int pix = py * cam.w + px;
  first[pix] = tf;
  thick[pix] = len;
  last[pix] = tl;
  if (visits) visits[pix] = nv;
}

// The site whose ball surface is nearest x, argmin |x - p| - r over the
// sites within `layers` grid cells (every site whose grown ball, radius
// r + grow, holds x is that near when layers covers r_max + grow); -1 and
// INFINITY when there is none.
__device__ int nearest_surface(const float* x, const V4<float>* __restrict__ sxp,
                               const int32_t* __restrict__ cell_start, const GridParams<float>& g,
                               int layers, float& dmin) {
  int c[3];
  for (int k = 0; k < 3; k++) c[k] = rcell(x[k], g.lo[k], g.inv_cs, g.dim[k]);
  float best = INFINITY;
  int besti = -1;
  for (int z = max(c[2] - layers, 0); z <= min(c[2] + layers, g.dim[2] - 1); z++)
    for (int y = max(c[1] - layers, 0); y <= min(c[1] + layers, g.dim[1] - 1); y++) {
      const int key0 = (z * g.dim[1] + y) * g.dim[0];
      const int a = cell_start[key0 + max(c[0] - layers, 0)];
      const int b = cell_start[key0 + min(c[0] + layers, g.dim[0] - 1) + 1];
      for (int s = a; s < b; s++) {
        const V4<float> p = sxp[s];
        if (!(p.w > 0.f)) continue;
        const float dx = x[0] - p.x, dy = x[1] - p.y, dz = x[2] - p.z;
        const float dist = sqrtf(dx * dx + dy * dy + dz * dz) - sqrtf(p.w);
        if (dist < best) {
          best = dist;
          besti = s;
        }
      }
    }
  dmin = best;
  return besti;
}

// Sphere tracing of the smoothed free surface (Sec. 6, surface smoothing).
// The signed distance of ball i is d_i(x) = |x - p_i| - r_i; at x the
// closest site i (nearest ball surface) and its Laguerre neighbourhood (the
// sites of its Hessian row: restricted facets above the emission
// threshold) give f = smin_k(d_(1), d_(2)), the cubic polynomial smooth
// union of the two nearest spheres of that set, smin_k(a, b) = min(a, b) -
// k h^3 / 6 with h = max(k - |a - b|, 0) / k.  f is 1-Lipschitz within one
// neighbourhood and f >= d_(1) - k/6, so the surface {f = 0} lies within
// k/6 of the balls: a ray point farther than that from every ball jumps to
// the next entry into the balls grown by k/6 (the grid walk), otherwise the
// march steps by f (at least kSmoothMinStep k) and stops at f <= kSmoothHit
// k.  Outputs per pixel: t of the hit (-1: none), the unit normal there
// (the smooth minimum's blend of the two spheres' normals; 0: none), and
// the evaluations taken (at most kSmoothMaxSteps).
constexpr float kSmoothHit = 1e-3f;
constexpr float kSmoothMinStep = 1e-4f;
constexpr int kSmoothMaxSteps = 1024;

__global__ void __launch_bounds__(128)
    k_render_smooth(Ray cam, Box<float> box, const V4<float>* __restrict__ sxp,
                    const int32_t* __restrict__ cell_start, GridParams<float> g, int layers,
                    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ cols,
                    float k, float* depth, float* normal, int32_t* steps) {
  const int px = blockIdx.x * blockDim.x + threadIdx.x;
  const int py = blockIdx.y * blockDim.y + threadIdx.y;
  if (px >= cam.w || py >= cam.h) return;
  float d[3];
  pixel_ray(cam, px, py, d);
  float t0, t1;
  box_span(box, cam.o, d, t0, t1);
  const float grow = k / 6.f;
  float t = t0, hit_t = -1.f;
  float nrm[3] = {0.f, 0.f, 0.f};
  int ns = 0;
  while (t <= t1 && ns < kSmoothMaxSteps) {
    ns++;
    const float x[3] = {cam.o[0] + t * d[0], cam.o[1] + t * d[1], cam.o[2] + t * d[2]};
    float d1;
    const int i = nearest_surface(x, sxp, cell_start, g, layers, d1);
    if (!(d1 <= grow)) {
      // farther than k/6 from every ball: the next entry into the grown balls
      int s = -1;
      const float te = next_entry(cam.o, d, t, t1, sxp, cell_start, g, layers,
                                  [](int) { return false; }, &s, grow);
      if (s < 0 || te > t1) break;
      if (te > t || i < 0) {
        t = fmaxf(te, t + kSmoothMinStep * k * (te > t ? 0.f : 1.f));
        continue;
      }
      // at the grown surface within rounding: a step of the march
    }
    const V4<float> p = sxp[i];
    float d2 = INFINITY;
    int j2 = -1;
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
      const int j = cols[e];
      const V4<float> q = sxp[j];
      if (!(q.w > 0.f)) continue;
      const float dx = x[0] - q.x, dy = x[1] - q.y, dz = x[2] - q.z;
      const float dj = sqrtf(dx * dx + dy * dy + dz * dz) - sqrtf(q.w);
      if (dj < d2) {
        d2 = dj;
        j2 = j;
      }
    }
    float f = d1, h = 0.f;
    if (j2 >= 0) {
      h = fmaxf(k - fabsf(d1 - d2), 0.f) / k;
      f = fminf(d1, d2) - k * h * h * h / 6.f;
    }
    if (f <= kSmoothHit * k) {
      hit_t = t;
      // d(smin)/da = 1 - h^2/2 for the smaller distance a, h^2/2 for the other
      const float wlo = 1.f - 0.5f * h * h;
      const float w1 = d1 <= d2 ? wlo : 1.f - wlo;
      float g1[3] = {x[0] - p.x, x[1] - p.y, x[2] - p.z};
      const float l1 = rsqrtf(g1[0] * g1[0] + g1[1] * g1[1] + g1[2] * g1[2]);
      for (int c = 0; c < 3; c++) nrm[c] = w1 * g1[c] * l1;
      if (j2 >= 0) {
        const V4<float> q = sxp[j2];
        float g2[3] = {x[0] - q.x, x[1] - q.y, x[2] - q.z};
        const float l2 = rsqrtf(g2[0] * g2[0] + g2[1] * g2[1] + g2[2] * g2[2]);
        for (int c = 0; c < 3; c++) nrm[c] += (1.f - w1) * g2[c] * l2;
      }
      const float ln = rsqrtf(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
      for (int c = 0; c < 3; c++) nrm[c] *= ln;
      break;
    }
    t += fmaxf(f, kSmoothMinStep * k);
  }
  const int pix = py * cam.w + px;
  depth[pix] = hit_t;
  if (normal)
    for (int c = 0; c < 3; c++) normal[3 * pix + c] = nrm[c];
  if (steps) steps[pix] = ns;
}

}  // namespace
}  // namespace pot

using namespace pot;

namespace {

// the camera's frame (right = forward x up, up' = right x forward)
int make_ray(const pot_camera* cam, Ray& ray) {
  if (cam->width <= 0 || cam->height <= 0 || !(cam->fov_y > 0.0 && cam->fov_y < 3.14))
    return POT_ERR_INVALID_ARG;
  double f[3], up[3], r[3], u[3];
  for (int k = 0; k < 3; k++) {
    f[k] = cam->forward[k];
    up[k] = cam->up[k];
  }
  const double fl = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  if (!(fl > 0.0)) return POT_ERR_INVALID_ARG;
  for (int k = 0; k < 3; k++) f[k] /= fl;
  r[0] = f[1] * up[2] - f[2] * up[1];
  r[1] = f[2] * up[0] - f[0] * up[2];
  r[2] = f[0] * up[1] - f[1] * up[0];
  const double rl = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  if (!(rl > 0.0)) return POT_ERR_INVALID_ARG;
  for (int k = 0; k < 3; k++) r[k] /= rl;
  u[0] = r[1] * f[2] - r[2] * f[1];
  u[1] = r[2] * f[0] - r[0] * f[2];
  u[2] = r[0] * f[1] - r[1] * f[0];
  for (int k = 0; k < 3; k++) {
    ray.o[k] = (float)cam->origin[k];
    ray.f[k] = (float)f[k];
    ray.r[k] = (float)r[k];
    ray.u[k] = (float)u[k];
  }
  ray.tv = (float)tan(0.5 * cam->fov_y);
  ray.th = ray.tv * (float)cam->width / (float)cam->height;
  ray.w = cam->width;
  ray.h = cam->height;
  return POT_OK;
}

}  // namespace

extern "C" int pot_render_depth(pot_ctx* ctx, void* stream, int64_t n, const float* pos,
                                const float* psi, const float* karea, const pot_domain* dom,
                                const pot_camera* cam, float* depth, float* normal) {
  if (!ctx || !pos || !psi || !dom || !cam || !depth || n <= 0 || n > ctx->n_max || !(ctx->mask & 1))
    return POT_ERR_INVALID_ARG;
  Ray ray;
  POT_CHECK(make_ray(cam, ray));
  if (cudaSetDevice(ctx->device) != cudaSuccess) return POT_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  POT_CHECK(grid_build<float>(ctx, st, n, pos, psi, nullptr, dom));
  Work<float>& w = ctx->wf;
  // ceil(r_max / cell) layers of neighbour cells (grid_build read psi_max)
  const double rmax = sqrt(fmax((double)*(float*)ctx->h_pinned, 0.0));
  const int layers = (int)fmax(1.0, ceil(rmax / (double)w.grid.cs));
  Box<float> box;
  for (int k = 0; k < 3; k++) {
    box.lo[k] = (float)dom->lo[k];
    box.hi[k] = (float)dom->hi[k];
  }
  dim3 blk(16, 16), grd((cam->width + 15) / 16, (cam->height + 15) / 16);
  note_launch();
  k_render<<<grd, blk, 0, st>>>(ray, box, w.sxp, ctx->perm, karea, ctx->cell_start, w.grid, layers,
                                depth, normal);
  POT_CUDA(cudaGetLastError());
  POT_CUDA(cudaStreamSynchronize(st));
  return POT_OK;
}

extern "C" int pot_render_volume(pot_ctx* ctx, void* stream, int64_t n, const float* pos,
                                 const float* psi, const pot_domain* dom, const pot_camera* cam,
                                 float* first, float* thickness, float* last, int32_t* visits) {
  if (!ctx || !pos || !psi || !dom || !cam || !first || !thickness || !last || n <= 0 ||
      n > ctx->n_max || !(ctx->mask & 1))
    return POT_ERR_INVALID_ARG;
  for (int k = 0; k < 3; k++)
    if (!(dom->hi[k] > dom->lo[k])) return POT_ERR_INVALID_ARG;
  Ray ray;
  POT_CHECK(make_ray(cam, ray));
  if (cudaSetDevice(ctx->device) != cudaSuccess) return POT_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  // the cells at these weights: their restricted facets (the Hessian rows'
  // columns, sorted space) and free-surface areas
  POT_CHECK(grid_build<float>(ctx, st, n, pos, psi, nullptr, dom));
  // ceil(r_max / cell) layers of neighbour cells (grid_build read psi_max)
  const double rmax = sqrt(fmax((double)*(float*)ctx->h_pinned, 0.0));
  Work<float>& w = ctx->wf;
  const int ce = cells_eval<float>(ctx, st, n, dom, false);
  int64_t site = -1;
  const int code = read_status(ctx, st, &site);
  if (code != POT_OK) return code;
  POT_CHECK(ce);
  int64_t nnz_off = 0;
  POT_CHECK(csr_compact<float>(ctx, st, n, &nnz_off));
  const int layers = (int)fmax(1.0, ceil(rmax / (double)w.grid.cs));
  Box<float> box;
  for (int k = 0; k < 3; k++) {
    box.lo[k] = (float)dom->lo[k];
    box.hi[k] = (float)dom->hi[k];
  }
  dim3 blk(16, 8), grd((cam->width + 15) / 16, (cam->height + 7) / 8);
  note_launch();
  k_render_volume<<<grd, blk, 0, st>>>(ray, box, w.sxp, w.karea, ctx->cell_start, w.grid, layers,
                                       ctx->row_ptr, ctx->csr_cols, first, thickness, last, visits);
  POT_CUDA(cudaGetLastError());
  POT_CUDA(cudaStreamSynchronize(st));
  return POT_OK;
}

extern "C" int pot_render_smooth(pot_ctx* ctx, void* stream, int64_t n, const float* pos,
                                 const float* psi, const pot_domain* dom, const pot_camera* cam,
                                 float k_smooth, float* depth, float* normal, int32_t* steps) {
  if (!ctx || !pos || !psi || !dom || !cam || !depth || n <= 0 || n > ctx->n_max ||
      !(ctx->mask & 1) || !(k_smooth > 0.f) || !isfinite(k_smooth))
    return POT_ERR_INVALID_ARG;
  for (int k = 0; k < 3; k++)
    if (!(dom->hi[k] > dom->lo[k])) return POT_ERR_INVALID_ARG;
  Ray ray;
  POT_CHECK(make_ray(cam, ray));
  if (cudaSetDevice(ctx->device) != cudaSuccess) return POT_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  // the cells at these weights: the Laguerre neighbourhoods are the Hessian
  // rows' columns (sorted space)
  POT_CHECK(grid_build<float>(ctx, st, n, pos, psi, nullptr, dom));
  const double rmax = sqrt(fmax((double)*(float*)ctx->h_pinned, 0.0));
  Work<float>& w = ctx->wf;
  const int ce = cells_eval<float>(ctx, st, n, dom, false);
  int64_t site = -1;
  const int code = read_status(ctx, st, &site);
  if (code != POT_OK) return code;
  POT_CHECK(ce);
  int64_t nnz_off = 0;
  POT_CHECK(csr_compact<float>(ctx, st, n, &nnz_off));
  // grid layers covering the grown balls, r_max + k/6
  const int layers =
      (int)fmax(1.0, ceil((rmax + (double)k_smooth / 6.0) / (double)w.grid.cs));
  Box<float> box;
  for (int k = 0; k < 3; k++) {
    box.lo[k] = (float)dom->lo[k];
    box.hi[k] = (float)dom->hi[k];
  }
  dim3 blk(16, 8), grd((cam->width + 15) / 16, (cam->height + 7) / 8);
  note_launch();
  k_render_smooth<<<grd, blk, 0, st>>>(ray, box, w.sxp, ctx->cell_start, w.grid, layers,
                                       ctx->row_ptr, ctx->csr_cols, k_smooth, depth, normal,
                                       steps);
  POT_CUDA(cudaGetLastError());
  POT_CUDA(cudaStreamSynchronize(st));
  return POT_OK;
}
