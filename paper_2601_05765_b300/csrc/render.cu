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

__global__ void __launch_bounds__(256)
    k_render(Ray cam, Box<float> box, const V4<float>* __restrict__ sxp,
             const int32_t* __restrict__ perm, const float* __restrict__ karea,
             const int32_t* __restrict__ cell_start, GridParams<float> g, int layers,
             float* depth, float* normal) {
  const int px = blockIdx.x * blockDim.x + threadIdx.x;
  const int py = blockIdx.y * blockDim.y + threadIdx.y;
  if (px >= cam.w || py >= cam.h) return;
  const float sx = ((px + 0.5f) / cam.w * 2.f - 1.f) * cam.th;
  const float sy = (1.f - (py + 0.5f) / cam.h * 2.f) * cam.tv;
  float d[3];
  for (int k = 0; k < 3; k++) d[k] = cam.f[k] + sx * cam.r[k] + sy * cam.u[k];
  const float il = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int k = 0; k < 3; k++) d[k] *= il;
  // the box along the ray: [t0, t1]
  float t0 = 0.f, t1 = INFINITY;
  for (int k = 0; k < 3; k++) {
    const float a = (box.lo[k] - cam.o[k]) / d[k], b = (box.hi[k] - cam.o[k]) / d[k];
    t0 = fmaxf(t0, fminf(a, b));
    t1 = fminf(t1, fmaxf(a, b));
  }
  float best = INFINITY;
  int besti = -1;
  if (t0 < t1) {
    int c[3], step[3];
    float tmax[3], tdel[3];
    for (int k = 0; k < 3; k++) {
      const float x = cam.o[k] + t0 * d[k];
      c[k] = rcell(x, g.lo[k], g.inv_cs, g.dim[k]);
      step[k] = d[k] > 0.f ? 1 : -1;
      const float edge = g.lo[k] + (c[k] + (d[k] > 0.f ? 1 : 0)) * g.cs;
      tmax[k] = d[k] != 0.f ? (edge - cam.o[k]) / d[k] : INFINITY;
      tdel[k] = d[k] != 0.f ? g.cs / fabsf(d[k]) : INFINITY;
    }
    float tcell = t0;
    while (tcell <= t1 && tcell <= best) {
      const int z0 = max(c[2] - layers, 0), z1 = min(c[2] + layers, g.dim[2] - 1);
      const int y0 = max(c[1] - layers, 0), y1 = min(c[1] + layers, g.dim[1] - 1);
      const int x0 = max(c[0] - layers, 0), x1 = min(c[0] + layers, g.dim[0] - 1);
      for (int z = z0; z <= z1; z++)
        for (int y = y0; y <= y1; y++) {
          const int key0 = (z * g.dim[1] + y) * g.dim[0];
          const int a = cell_start[key0 + x0], b = cell_start[key0 + x1 + 1];
          for (int s = a; s < b; s++) {
            const V4<float> p = sxp[s];
            if (!(p.w > 0.f)) continue;
            if (karea && !(karea[perm[s]] > 0.f)) continue;
            const float ex = p.x - cam.o[0], ey = p.y - cam.o[1], ez = p.z - cam.o[2];
            const float bb = ex * d[0] + ey * d[1] + ez * d[2];
            // r^2 minus the squared distance from the centre to the ray
            // (no cancellation between |e|^2 and b^2)
            const float hx = ex - bb * d[0], hy = ey - bb * d[1], hz = ez - bb * d[2];
            const float disc = p.w - (hx * hx + hy * hy + hz * hz);
            if (disc < 0.f) continue;
            const float sq = sqrtf(disc);
            const float t = fmaxf(bb - sq, t0);
            if (t < fminf(bb + sq, t1) && t < best) {
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

}  // namespace
}  // namespace pot

using namespace pot;

extern "C" int pot_render_depth(pot_ctx* ctx, void* stream, int64_t n, const float* pos,
                                const float* psi, const float* karea, const pot_domain* dom,
                                const pot_camera* cam, float* depth, float* normal) {
  if (!ctx || !pos || !psi || !dom || !cam || !depth || n <= 0 || n > ctx->n_max || !(ctx->mask & 1))
    return POT_ERR_INVALID_ARG;
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
  Ray ray;
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
