// capi.cu - operator entry points of the C ABI: A (Eq. 1), A^H (Eq. 2),
// A^H A (Section 2.1.5), their host-buffer forms and the stage calls.
#include <algorithm>
#include <cstdint>

#include "internal.cuh"

using namespace nufft;

namespace {

int check_plan(nufft_plan_t* p) {
  if (!p) return set_error(nullptr, NUFFT_EINVAL, "plan is NULL");
  return NUFFT_OK;
}

int check_ptr(nufft_plan_t* p, const void* ptr, int64_t count, const char* name) {
  if (count > 0 && !ptr) return set_error(p, NUFFT_EINVAL, "%s is NULL", name);
  return NUFFT_OK;
}

#define TRY(x)                 \
  do {                         \
    int _rc = (x);             \
    if (_rc != NUFFT_OK) return _rc; \
  } while (0)

int forward_impl(nufft_plan_t* p, const float2* x, float2* y) {
  if (p->M == 0) return NUFFT_OK;
  TRY(launch_fft_forward(p, x, p->grid));
  return launch_interp(p, p->grid, y);
}

int adjoint_impl(nufft_plan_t* p, const float2* y, float2* x) {
  TRY(launch_gridding(p, y, p->grid));
  return launch_fft_inverse(p, p->grid, x);
}

}  // namespace

namespace nufft {
// A^H A x, used by the solvers too.
int selfadjoint_impl(nufft_plan_t* p, const float2* x, float2* out) {
  TRY(launch_fft_forward(p, x, p->grid));
  if (vhv_fused(p)) {
    TRY(launch_vhv(p, p->grid, p->grid));     // gather then scatter per tile chunk
  } else {
    TRY(launch_interp(p, p->grid, p->ytmp));
    TRY(launch_gridding(p, p->ytmp, p->grid));
  }
  return launch_fft_inverse(p, p->grid, out);
}
int selfadjoint_hooked(nufft_plan_t* p, float2* x, float2* out, const CgHooks* h) {
  TRY(launch_fft_forward(p, x, p->grid, 1, true, h));
  if (vhv_fused(p)) {
    TRY(launch_vhv(p, p->grid, p->grid));
  } else {
    TRY(launch_interp(p, p->grid, p->ytmp));
    TRY(launch_gridding(p, p->ytmp, p->grid));
  }
  return launch_fft_inverse(p, p->grid, out, 1, true, h);
}
int forward_dev(nufft_plan_t* p, const float2* x, float2* y) { return forward_impl(p, x, y); }
int adjoint_dev(nufft_plan_t* p, const float2* y, float2* x) { return adjoint_impl(p, y, x); }

// Batched work space for nb transforms at once (grown on demand, kept).
int ensure_batch(nufft_plan_t* p, int nb) {
  if (nb <= p->batch_cap) return NUFFT_OK;
  drop_graphs(p);   // graphs may reference the buffers freed below
  for (float2** b : {&p->bgrid, &p->btiles, &p->bytmp, &p->bimg})
    if (*b) { dev_free(*b); *b = nullptr; }
  p->device_bytes -= (int64_t)p->batch_cap *
                     (p->Kprod + p->chunk_cap * p->g.padded_cells + (p->M > 0 ? p->M : 1) + p->Nprod) *
                     (int64_t)sizeof(float2);
  p->batch_cap = 0;
  const int64_t counts[4] = {(int64_t)nb * p->Kprod, (int64_t)nb * p->chunk_cap * p->g.padded_cells,
                             (int64_t)nb * (p->M > 0 ? p->M : 1), (int64_t)nb * p->Nprod};
  float2** bufs[4] = {&p->bgrid, &p->btiles, &p->bytmp, &p->bimg};
  for (int k = 0; k < 4; ++k) {
    if (counts[k] == 0) continue;
    cudaError_t e = dev_malloc((void**)bufs[k], counts[k] * sizeof(float2));
    if (e != cudaSuccess) {   // release what this call took; the plan keeps no batch capacity
      for (int q = 0; q < k; ++q)
        if (*bufs[q]) {
          dev_free(*bufs[q]);
          *bufs[q] = nullptr;
          p->device_bytes -= counts[q] * (int64_t)sizeof(float2);
        }
      *bufs[k] = nullptr;
      return cuda_check(p, e, "batched work space");
    }
    p->device_bytes += counts[k] * (int64_t)sizeof(float2);
  }
  p->batch_cap = nb;
  return NUFFT_OK;
}

// nb transforms: x is nb images, y is nb x M.
int forward_batch_impl(nufft_plan_t* p, int nb, const float2* x, float2* y) {
  if (nb == 1) return forward_impl(p, x, y);
  if (p->M == 0) return NUFFT_OK;
  TRY(ensure_batch(p, nb));
  TRY(launch_fft_forward(p, x, p->bgrid, nb));
  return launch_interp(p, p->bgrid, y, nb);
}

int adjoint_batch_impl(nufft_plan_t* p, int nb, const float2* y, float2* x) {
  if (nb == 1) return adjoint_impl(p, y, x);
  TRY(ensure_batch(p, nb));
  TRY(launch_gridding(p, y, p->bgrid, nb, p->btiles));
  return launch_fft_inverse(p, p->bgrid, x, nb);
}

int selfadjoint_batch_impl(nufft_plan_t* p, int nb, const float2* x, float2* out) {
  if (nb == 1) return selfadjoint_impl(p, x, out);
  TRY(ensure_batch(p, nb));
  TRY(launch_fft_forward(p, x, p->bgrid, nb));
  // V then V^H: for a batch (the coils of multi-coil operators) the separate
  // passes measured ~3% faster than the fused one, which wins for one transform
  TRY(launch_interp(p, p->bgrid, p->bytmp, nb));
  TRY(launch_gridding(p, p->bytmp, p->bgrid, nb, p->btiles));
  return launch_fft_inverse(p, p->bgrid, out, nb);
}
}  // namespace nufft

extern "C" int nufft_forward(nufft_plan_t* p, const float* x_dev, float* y_dev) {
  TRY(check_plan(p));
  TRY(check_ptr(p, x_dev, p->Nprod, "x_dev"));
  TRY(check_ptr(p, y_dev, p->M, "y_dev"));
  const float2* x = reinterpret_cast<const float2*>(x_dev);
  float2* y = reinterpret_cast<float2*>(y_dev);
  return run_graphed(p, 1, x, y, 0, [&]() { return forward_impl(p, x, y); });
}

extern "C" int nufft_adjoint(nufft_plan_t* p, const float* y_dev, float* x_dev) {
  TRY(check_plan(p));
  TRY(check_ptr(p, y_dev, p->M, "y_dev"));
  TRY(check_ptr(p, x_dev, p->Nprod, "x_dev"));
  const float2* y = reinterpret_cast<const float2*>(y_dev);
  float2* x = reinterpret_cast<float2*>(x_dev);
  return run_graphed(p, 2, y, x, 0, [&]() { return adjoint_impl(p, y, x); });
}

extern "C" int nufft_selfadjoint(nufft_plan_t* p, const float* x_dev, float* out_dev) {
  TRY(check_plan(p));
  TRY(check_ptr(p, x_dev, p->Nprod, "x_dev"));
  TRY(check_ptr(p, out_dev, p->Nprod, "out_dev"));
  if ((const void*)x_dev == (const void*)out_dev) return set_error(p, NUFFT_EINVAL, "x_dev and out_dev alias");
  const float2* x = reinterpret_cast<const float2*>(x_dev);
  float2* out = reinterpret_cast<float2*>(out_dev);
  return run_graphed(p, 3, x, out, 0, [&]() { return selfadjoint_impl(p, x, out); });
}

namespace {
// Copies between device memory and the device alias of page-locked host
// memory, run by the SMs: many 16-byte accesses in flight cross NVLink-C2C
// faster than a copy-engine transfer of the same ~MB size.
__global__ void k_copy16(const float4* __restrict__ src, float4* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}
__global__ void k_copy8(const float2* __restrict__ src, float2* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

int sm_copy(nufft_plan_t* p, const float2* src, float2* dst, int64_t n) {
  if (n == 0) return NUFFT_OK;
  const bool v16 = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) % 16 == 0) && n % 2 == 0;
  const int64_t items = v16 ? n / 2 : n;
  const int64_t blocks = std::min<int64_t>((items + 255) / 256, 152 * 8);
  if (v16)
    k_copy16<<<(unsigned)blocks, 256, 0, p->stream>>>(reinterpret_cast<const float4*>(src),
                                                        reinterpret_cast<float4*>(dst), items);
  else
    k_copy8<<<(unsigned)blocks, 256, 0, p->stream>>>(src, dst, items);
  NUFFT_CUDA_TRY(p, cudaGetLastError());
  return NUFFT_OK;
}

// The device address of page-locked (cudaHostAlloc / cudaHostRegister) host
// memory, or nullptr for any other memory.
void* device_alias(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}
}  // namespace

extern "C" int nufft_forward_host(nufft_plan_t* p, const float* x_host, float* y_host) {
  TRY(check_plan(p));
  TRY(check_ptr(p, x_host, p->Nprod, "x_host"));
  TRY(check_ptr(p, y_host, p->M, "y_host"));
  // Page-locked buffers: the first FFT pass reads the image straight from host
  // memory, the samples go back by an SM copy through the host alias, and the
  // whole sequence is recorded as one graph per buffer pair.  Other host
  // memory goes through the staging buffers eagerly, so a recorded access
  // never meets memory that is no longer page-locked (checked on every call).
  const float2* x_alias = static_cast<const float2*>(device_alias(x_host));
  float2* y_alias = static_cast<float2*>(device_alias(y_host));
  const bool locked = x_alias && (p->M == 0 || y_alias);
  auto body = [&]() -> int {
    const float2* x = x_alias;
    if (!locked) {
      NUFFT_CUDA_TRY(p, cudaMemcpyAsync(p->x_stage, x_host, p->Nprod * sizeof(float2), cudaMemcpyHostToDevice,
                                        p->stream));
      x = p->x_stage;
    }
    TRY(forward_impl(p, x, p->y_stage));
    if (p->M > 0) {
      if (locked) TRY(sm_copy(p, p->y_stage, y_alias, p->M));
      else NUFFT_CUDA_TRY(p, cudaMemcpyAsync(y_host, p->y_stage, p->M * sizeof(float2), cudaMemcpyDeviceToHost,
                                             p->stream));
    }
    return NUFFT_OK;
  };
  if (locked) TRY(run_graphed(p, 21, x_host, y_host, 0, body));
  else TRY(body());
  NUFFT_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
  return NUFFT_OK;
}

extern "C" int nufft_adjoint_host(nufft_plan_t* p, const float* y_host, float* x_host) {
  TRY(check_plan(p));
  TRY(check_ptr(p, y_host, p->M, "y_host"));
  TRY(check_ptr(p, x_host, p->Nprod, "x_host"));
  // Page-locked buffers: the samples come up by an SM copy through the host
  // alias and the last inverse FFT pass writes the image straight to host
  // memory (see the forward form).
  float2* x_alias = static_cast<float2*>(device_alias(x_host));
  const float2* y_alias = static_cast<const float2*>(device_alias(y_host));
  const bool locked = x_alias && (p->M == 0 || y_alias);
  auto body = [&]() -> int {
    if (p->M > 0) {
      if (locked) TRY(sm_copy(p, y_alias, p->y_stage, p->M));
      else NUFFT_CUDA_TRY(p, cudaMemcpyAsync(p->y_stage, y_host, p->M * sizeof(float2), cudaMemcpyHostToDevice,
                                             p->stream));
    }
    if (locked) return adjoint_impl(p, p->y_stage, x_alias);
    TRY(adjoint_impl(p, p->y_stage, p->x_stage));
    NUFFT_CUDA_TRY(p, cudaMemcpyAsync(x_host, p->x_stage, p->Nprod * sizeof(float2), cudaMemcpyDeviceToHost, p->stream));
    return NUFFT_OK;
  };
  if (locked) TRY(run_graphed(p, 22, y_host, x_host, 0, body));
  else TRY(body());
  NUFFT_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
  return NUFFT_OK;
}

extern "C" int nufft_scale_pad_fft(nufft_plan_t* p, const float* x_dev, float* grid_dev) {
  TRY(check_plan(p));
  TRY(check_ptr(p, x_dev, p->Nprod, "x_dev"));
  TRY(check_ptr(p, grid_dev, p->Kprod, "grid_dev"));
  const float2* x = reinterpret_cast<const float2*>(x_dev);
  float2* grid = reinterpret_cast<float2*>(grid_dev);
  return run_graphed(p, 11, x, grid, 0, [&]() { return launch_fft_forward(p, x, grid); });
}

extern "C" int nufft_interp(nufft_plan_t* p, const float* grid_dev, float* y_dev) {
  TRY(check_plan(p));
  TRY(check_ptr(p, grid_dev, p->Kprod, "grid_dev"));
  TRY(check_ptr(p, y_dev, p->M, "y_dev"));
  const float2* grid = reinterpret_cast<const float2*>(grid_dev);
  float2* y = reinterpret_cast<float2*>(y_dev);
  return run_graphed(p, 12, grid, y, 0, [&]() { return launch_interp(p, grid, y); });
}

extern "C" int nufft_gridding(nufft_plan_t* p, const float* y_dev, float* grid_dev) {
  TRY(check_plan(p));
  TRY(check_ptr(p, y_dev, p->M, "y_dev"));
  TRY(check_ptr(p, grid_dev, p->Kprod, "grid_dev"));
  const float2* y = reinterpret_cast<const float2*>(y_dev);
  float2* grid = reinterpret_cast<float2*>(grid_dev);
  return run_graphed(p, 13, y, grid, 0, [&]() { return launch_gridding(p, y, grid); });
}

extern "C" int nufft_ifft_crop_rescale(nufft_plan_t* p, float* grid_dev, float* x_dev) {
  TRY(check_plan(p));
  TRY(check_ptr(p, grid_dev, p->Kprod, "grid_dev"));
  TRY(check_ptr(p, x_dev, p->Nprod, "x_dev"));
  float2* grid = reinterpret_cast<float2*>(grid_dev);
  float2* x = reinterpret_cast<float2*>(x_dev);
  return run_graphed(p, 14, grid, x, 0, [&]() { return launch_fft_inverse(p, grid, x); });
}

extern "C" int nufft_forward_batch(nufft_plan_t* p, int nb, const float* x_dev, float* y_dev) {
  TRY(check_plan(p));
  if (nb < 1) return set_error(p, NUFFT_EINVAL, "nb < 1");
  TRY(check_ptr(p, x_dev, p->Nprod, "x_dev"));
  TRY(check_ptr(p, y_dev, p->M, "y_dev"));
  const float2* x = reinterpret_cast<const float2*>(x_dev);
  float2* y = reinterpret_cast<float2*>(y_dev);
  return run_graphed(p, 4, x, y, nb, [&]() { return forward_batch_impl(p, nb, x, y); });
}

extern "C" int nufft_adjoint_batch(nufft_plan_t* p, int nb, const float* y_dev, float* x_dev) {
  TRY(check_plan(p));
  if (nb < 1) return set_error(p, NUFFT_EINVAL, "nb < 1");
  TRY(check_ptr(p, y_dev, p->M, "y_dev"));
  TRY(check_ptr(p, x_dev, p->Nprod, "x_dev"));
  const float2* y = reinterpret_cast<const float2*>(y_dev);
  float2* x = reinterpret_cast<float2*>(x_dev);
  return run_graphed(p, 5, y, x, nb, [&]() { return adjoint_batch_impl(p, nb, y, x); });
}

extern "C" int nufft_selfadjoint_batch(nufft_plan_t* p, int nb, const float* x_dev, float* out_dev) {
  TRY(check_plan(p));
  if (nb < 1) return set_error(p, NUFFT_EINVAL, "nb < 1");
  TRY(check_ptr(p, x_dev, p->Nprod, "x_dev"));
  TRY(check_ptr(p, out_dev, p->Nprod, "out_dev"));
  if ((const void*)x_dev == (const void*)out_dev) return set_error(p, NUFFT_EINVAL, "x_dev and out_dev alias");
  const float2* x = reinterpret_cast<const float2*>(x_dev);
  float2* out = reinterpret_cast<float2*>(out_dev);
  return run_graphed(p, 6, x, out, nb, [&]() { return selfadjoint_batch_impl(p, nb, x, out); });
}
