// grad.cu - gradient of the forward NUFFT with respect to the trajectory.
//
// y_m = sum_j prod_d c_{m,d,j_d}(w_m) Y[k0_m + j] with Y = F S x (Section 2.1,
// Eq. 1; Section 2.1.3).  The neighbourhood k0 is piecewise constant in w,
// so inside a cell
//   d y_m / d w_{m,a} = sum_j (d c_{m,a,j_a} / d w) prod_{d != a} c_{m,d,j_d} Y[k0_m + j],
// with d c / d w = G^{-1} d r / d w from the min-max construction.  For a real
// loss with g = dL/dRe(y) + i dL/dIm(y), dL/dw_{m,a} = Re(conj(g_m) dy_m/dw_{m,a}).
// The kernel follows the interpolation kernel's lane layout (J_last lanes per
// point) and accumulates the value and the d derivative partials from the same
// grid loads.
#include "internal.cuh"

namespace nufft {
namespace {

struct GradView {
  const float2* dcoef;   // same layout as Points::coef
};

template <int D, int JF>
__global__ void __launch_bounds__(256)
k_traj_grad(const float2* __restrict__ grid, const float2* __restrict__ gy, float* __restrict__ gom, const Points P,
            const GradView Dv, const Geom g) {
  const int G = JF > 0 ? JF : g.J[D - 1];
  const int lane = threadIdx.x & 31;
  const int per_warp = 32 / G;
  const int sub = lane / G;
  const int l = lane - sub * G;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t i = warp * per_warp + sub;
  const bool active = (sub < per_warp) && (i < P.M);

  float2 part[D];  // partial d y / d w_a for a = 0..D-1
#pragma unroll
  for (int a = 0; a < D; ++a) part[a] = make_float2(0.f, 0.f);
  if (active) {
    const int kl = P.kf[(int64_t)(D - 1) * P.M + i];
    const int gl = wrapk(kl + l, g.K[D - 1]);
    const int64_t cl_idx = P.coef_off[D - 1] + (int64_t)l * P.M + i;
    const float2 cl = P.coef[cl_idx];
    const float2 dcl = Dv.dcoef[cl_idx];
    if (D == 1) {
      part[0] = cmul(dcl, __ldg(&grid[gl]));
    } else if (D == 2) {
      const int J0 = JF > 0 ? JF : g.J[0];
      const int k0 = P.kf[i];
      float2 acc_c = make_float2(0.f, 0.f), acc_d = make_float2(0.f, 0.f);
      for (int j0 = 0; j0 < J0; ++j0) {
        const int64_t ci = P.coef_off[0] + (int64_t)j0 * P.M + i;
        const float2 v = __ldg(&grid[wrapk(k0 + j0, g.K[0]) * (int)g.Kstride[0] + gl]);
        acc_c = cadd(acc_c, cmul(P.coef[ci], v));
        acc_d = cadd(acc_d, cmul(Dv.dcoef[ci], v));
      }
      part[0] = cmul(cl, acc_d);
      part[D - 1] = cmul(dcl, acc_c);
    } else {
      const int J0 = JF > 0 ? JF : g.J[0];
      const int J1 = JF > 0 ? JF : g.J[1];
      const int k0 = P.kf[i], k1 = P.kf[P.M + i];
      float2 acc_cc = make_float2(0.f, 0.f), acc_dc = make_float2(0.f, 0.f), acc_cd = make_float2(0.f, 0.f);
      for (int j0 = 0; j0 < J0; ++j0) {
        const int64_t c0i = P.coef_off[0] + (int64_t)j0 * P.M + i;
        const float2 c0 = P.coef[c0i], dc0 = Dv.dcoef[c0i];
        const float2* plane = grid + wrapk(k0 + j0, g.K[0]) * (int)g.Kstride[0];
        float2 s_c = make_float2(0.f, 0.f), s_d = make_float2(0.f, 0.f);
        for (int j1 = 0; j1 < J1; ++j1) {
          const int64_t c1i = P.coef_off[1] + (int64_t)j1 * P.M + i;
          const float2 v = __ldg(&plane[wrapk(k1 + j1, g.K[1]) * (int)g.Kstride[1] + gl]);
          s_c = cadd(s_c, cmul(P.coef[c1i], v));
          s_d = cadd(s_d, cmul(Dv.dcoef[c1i], v));
        }
        acc_cc = cadd(acc_cc, cmul(c0, s_c));
        acc_dc = cadd(acc_dc, cmul(dc0, s_c));
        acc_cd = cadd(acc_cd, cmul(c0, s_d));
      }
      part[0] = cmul(cl, acc_dc);
      part[1] = cmul(cl, acc_cd);
      part[2] = cmul(dcl, acc_cc);
    }
  }
  const int base = sub * G;
  float2 tot[D];
#pragma unroll
  for (int a = 0; a < D; ++a) tot[a] = make_float2(0.f, 0.f);
  for (int q = 0; q < G; ++q) {
    const int src = (base + q) & 31;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      tot[a].x += __shfl_sync(0xffffffffu, part[a].x, src);
      tot[a].y += __shfl_sync(0xffffffffu, part[a].y, src);
    }
  }
  if (active && l == 0) {
    const int64_t m = P.perm[i];
    const float2 gm = gy[m];
#pragma unroll
    for (int a = 0; a < D; ++a) gom[m * D + a] = gm.x * tot[a].x + gm.y * tot[a].y;  // Re(conj(g) dy)
  }
}

bool all_j6(const Geom& g) {
  for (int a = 0; a < g.d; ++a)
    if (g.J[a] != 6) return false;
  return true;
}

template <int D>
cudaError_t traj_grad_d(const nufft_plan_t* p, const float2* grid, const float2* gy, float* gom) {
  const Points P = points_view(p);
  GradView Dv;
  Dv.dcoef = p->dcoef;
  const int per_warp = 32 / p->g.J[D - 1];
  const int64_t warps = (P.M + per_warp - 1) / per_warp;
  const int64_t blocks = (warps * 32 + 255) / 256;
  if (blocks == 0) return cudaSuccess;
  if (all_j6(p->g)) k_traj_grad<D, 6><<<(unsigned)blocks, 256, 0, p->stream>>>(grid, gy, gom, P, Dv, p->g);
  else k_traj_grad<D, 0><<<(unsigned)blocks, 256, 0, p->stream>>>(grid, gy, gom, P, Dv, p->g);
  return cudaGetLastError();
}

}  // namespace
}  // namespace nufft

using namespace nufft;

extern "C" int nufft_trajectory_gradient(nufft_plan_t* p, const float* x_dev, const float* g_dev, float* gom_dev) {
  if (!p) return set_error(nullptr, NUFFT_EINVAL, "plan is NULL");
  if (!x_dev || (p->M > 0 && (!g_dev || !gom_dev)))
    return set_error(p, NUFFT_EINVAL, "x_dev, g_dev or gom_dev is NULL");
  if (p->M == 0) return NUFFT_OK;
  int rc = ensure_coef_derivatives(p);   // lazily, before any recording
  if (rc != NUFFT_OK) return rc;
  const float2* gy = reinterpret_cast<const float2*>(g_dev);
  return run_graphed(p, 23, x_dev, gom_dev, graph_key({graph_bits(g_dev)}), [&]() -> int {
    int r = launch_fft_forward(p, reinterpret_cast<const float2*>(x_dev), p->grid);
    if (r != NUFFT_OK) return r;
    cudaError_t e;
    switch (p->g.d) {
      case 1: e = traj_grad_d<1>(p, p->grid, gy, gom_dev); break;
      case 2: e = traj_grad_d<2>(p, p->grid, gy, gom_dev); break;
      default: e = traj_grad_d<3>(p, p->grid, gy, gom_dev); break;
    }
    return e == cudaSuccess ? NUFFT_OK : cuda_check(p, e, "trajectory gradient kernel");
  });
}

extern "C" int nufft_trajectory_gradient_grid(nufft_plan_t* p, const float* grid_dev, const float* g_dev,
                                              float* gom_dev) {
  if (!p) return set_error(nullptr, NUFFT_EINVAL, "plan is NULL");
  if (!grid_dev || (p->M > 0 && (!g_dev || !gom_dev)))
    return set_error(p, NUFFT_EINVAL, "grid_dev, g_dev or gom_dev is NULL");
  if (p->M == 0) return NUFFT_OK;
  int rc = ensure_coef_derivatives(p);
  if (rc != NUFFT_OK) return rc;
  const float2* grid = reinterpret_cast<const float2*>(grid_dev);
  const float2* gy = reinterpret_cast<const float2*>(g_dev);
  return run_graphed(p, 24, grid_dev, gom_dev, graph_key({graph_bits(g_dev)}), [&]() -> int {
    cudaError_t e;
    switch (p->g.d) {
      case 1: e = traj_grad_d<1>(p, grid, gy, gom_dev); break;
      case 2: e = traj_grad_d<2>(p, grid, gy, gom_dev); break;
      default: e = traj_grad_d<3>(p, grid, gy, gom_dev); break;
    }
    return e == cudaSuccess ? NUFFT_OK : cuda_check(p, e, "trajectory gradient kernel");
  });
}
