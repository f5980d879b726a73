// recon.cu - density compensation and multi-coil operators.
//
// Section 2.2.1 (Eqs. 5-6): sampling density compensation by the Pipe-Menon
// iteration w <- w / (A A^H w) and the gridding reconstruction
// x = A^H (y . w).  A A^H w is complex for real w (the centred grid gives the
// point-spread function a half-sample phase); the update divides by its
// magnitude, which keeps w real and positive.
// Section 2.2.3 (Eqs. 32-33): multi-coil operators A_i x = A (c_i . x) and
// A_multi^H A_multi x = sum_i conj(c_i) . A^H A (c_i . x).  All coils run as
// one batch of the NUFFT kernels (one launch per stage), between one kernel
// that forms every coil image and one that sums the conjugate-weighted coils.
#include <initializer_list>
#include <utility>

#include "internal.cuh"

namespace nufft {
int forward_dev(nufft_plan_t* p, const float2* x, float2* y);
int adjoint_dev(nufft_plan_t* p, const float2* y, float2* x);
int selfadjoint_impl(nufft_plan_t* p, const float2* x, float2* out);

namespace {

constexpr int kThreads = 256;

int blocks_for(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

__global__ void k_real_to_complex(const float* w, float2* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_float2(w[i], 0.f);
}

// w <- w / |d|  (a point whose |d| is 0 keeps its weight)
__global__ void k_dcf_update(float* w, const float2* d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = d[i];
    const float mag = sqrtf(v.x * v.x + v.y * v.y);
    if (mag > 0.f) w[i] = w[i] / mag;
  }
}

__global__ void k_weight(const float2* y, const float* w, float2* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = cscale(y[i], w[i]);
}

// out[b] = c[b] . x for all nc coils (nc x n outputs)
__global__ void k_coil_mul_all(const float2* c, const float2* x, float2* out, int64_t n, int nc) {
  const int64_t tot = n * nc;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < tot; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = cmul(c[k], x[k % n]);
}

// out = sum_b conj(c[b]) . v[b], coils summed in order b = 0..nc-1
__global__ void k_coil_conj_reduce(const float2* c, const float2* v, float2* out, int64_t n, int nc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (int b = 0; b < nc; ++b) acc = cadd(acc, cmulc(c[(int64_t)b * n + i], v[(int64_t)b * n + i]));
    out[i] = acc;
  }
}

#define TRY(x)                       \
  do {                               \
    int _rc = (x);                   \
    if (_rc != NUFFT_OK) return _rc; \
  } while (0)

}  // namespace

// Auxiliary buffers: two M-sized and two image-sized complex vectors.
int get_aux(nufft_plan_t* p, float2** m0, float2** m1, float2** i0, float2** i1) {
  const int64_t M = p->M > 0 ? p->M : 1;
  if (!p->mbuf) {
    const int64_t count = 2 * M + 2 * p->Nprod;
    cudaError_t e = dev_malloc((void**)&p->mbuf, count * sizeof(float2));
    if (e != cudaSuccess) {
      p->mbuf = nullptr;
      return cuda_check(p, e, "auxiliary work space");
    }
    p->device_bytes += count * (int64_t)sizeof(float2);
  }
  *m0 = p->mbuf;
  *m1 = p->mbuf + M;
  *i0 = p->mbuf + 2 * M;
  *i1 = p->mbuf + 2 * M + p->Nprod;
  return NUFFT_OK;
}

// All coils of the operator run as one batch: one coil-multiply kernel, one
// launch per NUFFT stage for the nc transforms, one conjugate-coil reduction.
int selfadjoint_multicoil_impl(nufft_plan_t* p, const float2* coils, int nc, const float2* x, float2* out) {
  const int64_t n = p->Nprod;
  float2 *imgs, *res;      // coil images in, A^H A of each coil image out
  if (nc == 1) {
    float2 *m0 = nullptr, *m1 = nullptr, *i0 = nullptr, *i1 = nullptr;
    TRY(get_aux(p, &m0, &m1, &i0, &i1));
    imgs = i0;
    res = i1;
  } else {
    TRY(ensure_batch(p, nc));
    imgs = res = p->bimg;  // the batched operator reads its input before writing its output
  }
  k_coil_mul_all<<<blocks_for(n * nc), kThreads, 0, p->stream>>>(coils, x, imgs, n, nc);
  NUFFT_CUDA_TRY(p, cudaGetLastError());
  TRY(normal_op(p, imgs, res, nc));
  k_coil_conj_reduce<<<blocks_for(n), kThreads, 0, p->stream>>>(coils, res, out, n, nc);
  NUFFT_CUDA_TRY(p, cudaGetLastError());
  return NUFFT_OK;
}

int adjoint_multicoil_impl(nufft_plan_t* p, const float2* coils, int nc, const float2* y, float2* x) {
  float2* imgs;
  if (nc == 1) {
    float2 *m0 = nullptr, *m1 = nullptr, *i0 = nullptr, *i1 = nullptr;
    TRY(get_aux(p, &m0, &m1, &i0, &i1));
    imgs = i0;
  } else {
    TRY(ensure_batch(p, nc));
    imgs = p->bimg;
  }
  TRY(adjoint_batch_impl(p, nc, y, imgs));
  k_coil_conj_reduce<<<blocks_for(p->Nprod), kThreads, 0, p->stream>>>(coils, imgs, x, p->Nprod, nc);
  NUFFT_CUDA_TRY(p, cudaGetLastError());
  return NUFFT_OK;
}

}  // namespace nufft

using namespace nufft;

namespace {
int check_plan_ptrs(nufft_plan_t* p, std::initializer_list<std::pair<const void*, int64_t>> ptrs) {
  if (!p) return set_error(nullptr, NUFFT_EINVAL, "plan is NULL");
  for (auto& pr : ptrs)
    if (pr.second > 0 && !pr.first) return set_error(p, NUFFT_EINVAL, "a required buffer is NULL");
  return NUFFT_OK;
}
}  // namespace

extern "C" int nufft_density_compensation(nufft_plan_t* p, float* w_dev, int iters) {
  TRY(check_plan_ptrs(p, {{w_dev, p ? p->M : 0}}));
  if (iters < 0) return set_error(p, NUFFT_EINVAL, "iters < 0");
  if (p->M == 0) return NUFFT_OK;
  float2 *m0 = nullptr, *m1 = nullptr, *i0 = nullptr, *i1 = nullptr;
  TRY(get_aux(p, &m0, &m1, &i0, &i1));
  return run_graphed(p, 19, w_dev, nullptr, iters, [&]() -> int {
    for (int it = 0; it < iters; ++it) {
      k_real_to_complex<<<blocks_for(p->M), kThreads, 0, p->stream>>>(w_dev, m0, p->M);
      NUFFT_CUDA_TRY(p, cudaGetLastError());
      TRY(adjoint_dev(p, m0, i0));
      TRY(forward_dev(p, i0, m1));
      k_dcf_update<<<blocks_for(p->M), kThreads, 0, p->stream>>>(w_dev, m1, p->M);
      NUFFT_CUDA_TRY(p, cudaGetLastError());
    }
    return NUFFT_OK;
  });
}

extern "C" int nufft_gridding_recon(nufft_plan_t* p, const float* y_dev, const float* w_dev, float* x_dev) {
  TRY(check_plan_ptrs(p, {{y_dev, p ? p->M : 0}, {w_dev, p ? p->M : 0}, {x_dev, p ? p->Nprod : 0}}));
  float2 *m0 = nullptr, *m1 = nullptr, *i0 = nullptr, *i1 = nullptr;
  TRY(get_aux(p, &m0, &m1, &i0, &i1));
  return run_graphed(p, 20, y_dev, x_dev, graph_key({graph_bits(w_dev)}), [&]() -> int {
    if (p->M > 0) {
      k_weight<<<blocks_for(p->M), kThreads, 0, p->stream>>>(reinterpret_cast<const float2*>(y_dev), w_dev, m0, p->M);
      NUFFT_CUDA_TRY(p, cudaGetLastError());
    }
    return adjoint_dev(p, m0, reinterpret_cast<float2*>(x_dev));
  });
}

extern "C" int nufft_forward_multicoil(nufft_plan_t* p, const float* coils_dev, int nc, const float* x_dev,
                                       float* y_dev) {
  TRY(check_plan_ptrs(p, {{coils_dev, p ? p->Nprod : 0}, {x_dev, p ? p->Nprod : 0}, {y_dev, p ? p->M : 0}}));
  if (nc < 1) return set_error(p, NUFFT_EINVAL, "nc < 1");
  float2* imgs;
  if (nc == 1) {
    float2 *m0 = nullptr, *m1 = nullptr, *i0 = nullptr, *i1 = nullptr;
    TRY(get_aux(p, &m0, &m1, &i0, &i1));
    imgs = i0;
  } else {
    TRY(ensure_batch(p, nc));
    imgs = p->bimg;
  }
  const int64_t n = p->Nprod;
  return run_graphed(p, 16, x_dev, y_dev, graph_key({graph_bits(coils_dev), (uint64_t)nc}), [&]() -> int {
    k_coil_mul_all<<<blocks_for(n * nc), kThreads, 0, p->stream>>>(reinterpret_cast<const float2*>(coils_dev),
                                                                   reinterpret_cast<const float2*>(x_dev), imgs, n, nc);
    NUFFT_CUDA_TRY(p, cudaGetLastError());
    return forward_batch_impl(p, nc, imgs, reinterpret_cast<float2*>(y_dev));
  });
}

extern "C" int nufft_adjoint_multicoil(nufft_plan_t* p, const float* coils_dev, int nc, const float* y_dev,
                                       float* x_dev) {
  TRY(check_plan_ptrs(p, {{coils_dev, p ? p->Nprod : 0}, {y_dev, p ? p->M : 0}, {x_dev, p ? p->Nprod : 0}}));
  if (nc < 1) return set_error(p, NUFFT_EINVAL, "nc < 1");
  return run_graphed(p, 17, y_dev, x_dev, graph_key({graph_bits(coils_dev), (uint64_t)nc}), [&]() {
    return adjoint_multicoil_impl(p, reinterpret_cast<const float2*>(coils_dev), nc,
                                  reinterpret_cast<const float2*>(y_dev), reinterpret_cast<float2*>(x_dev));
  });
}

extern "C" int nufft_selfadjoint_multicoil(nufft_plan_t* p, const float* coils_dev, int nc, const float* x_dev,
                                           float* out_dev) {
  TRY(check_plan_ptrs(p, {{coils_dev, p ? p->Nprod : 0}, {x_dev, p ? p->Nprod : 0}, {out_dev, p ? p->Nprod : 0}}));
  if (nc < 1) return set_error(p, NUFFT_EINVAL, "nc < 1");
  if ((const void*)x_dev == (const void*)out_dev) return set_error(p, NUFFT_EINVAL, "x_dev and out_dev alias");
  return run_graphed(p, 18, x_dev, out_dev, graph_key({graph_bits(coils_dev), (uint64_t)nc}), [&]() {
    return selfadjoint_multicoil_impl(p, reinterpret_cast<const float2*>(coils_dev), nc,
                                      reinterpret_cast<const float2*>(x_dev), reinterpret_cast<float2*>(out_dev));
  });
}
