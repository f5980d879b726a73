// toeplitz.cu - Toeplitz-embedded normal operator A^H A.
//
// Section 2.1.5: iterative solvers apply the normal operator A^H A, and the
// paper precomputes it (citing Fessler et al.'s Toeplitz method).  With
// t_n = n - N/2,
//   (A^H A x)[n] = sum_n' x[n'] t[n - n'],   t[D] = sum_m exp(i w_m . D),
// a convolution with t on D in (-N, N)^d.  Embedded circularly in a grid of
// period P >= 2N (2N rounded up to a power of two),
// A^H A x = crop(F^{-1}(T . F zero-pad(x))) with T the DFT of the circular t.
// The kernel t is the adjoint NUFFT of all-ones on an image of size P (grid
// 2P, same J), so it carries the NUFFT's accuracy (~1e-6 relative).  Each
// application is then a pruned FFT on the P grid, a pointwise product and a
// pruned inverse FFT: no interpolation or gridding per solver iteration.
#include "internal.cuh"

namespace nufft {
int selfadjoint_batch_impl(nufft_plan_t* p, int nb, const float2* x, float2* out);

namespace {

constexpr int kThreads = 256;

int nblocks(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

// om_rows[m * d + a] = om_sorted[a * M + m]   (point order is irrelevant here)
__global__ void k_om_rows(const float* om_sorted, int64_t M, int d, float* om_rows) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < M * d; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = k / d;
    const int a = (int)(k - m * d);
    om_rows[k] = om_sorted[(int64_t)a * M + m];
  }
}

__global__ void k_fill(float2* v, int64_t n, float2 val) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = val;
}

__global__ void k_scale(float2* v, int64_t n, float s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = cscale(v[i], s);
}

// grid[b][i] *= T[i] for every batch element b
__global__ void k_mul_spectrum(float2* grid, const float2* T, int64_t n, int nb) {
  const int64_t tot = n * nb;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < tot; k += (int64_t)gridDim.x * blockDim.x)
    grid[k] = cmul(grid[k], T[k % n]);
}

#define TRY(x)                       \
  do {                               \
    int _rc = (x);                   \
    if (_rc != NUFFT_OK) return _rc; \
  } while (0)

struct DevBuf {
  void* ptr = nullptr;
  ~DevBuf() { if (ptr) dev_free(ptr); }
};
struct PlanGuard {
  nufft_plan_t* p = nullptr;
  ~PlanGuard() { if (p) nufft_plan_destroy(p); }
};

int toeplitz_apply(nufft_plan_t* p, const float2* x, float2* out, int nb, const CgHooks* h = nullptr) {
  nufft_plan_t* tg = p->toep_geom;
  if (nb > p->toep_cap) {
    drop_graphs(p);   // graphs may reference the buffer freed below
    if (p->toep_grid) dev_free(p->toep_grid);
    p->toep_grid = nullptr;
    p->toep_cap = 0;
    NUFFT_CUDA_TRY(p, dev_malloc((void**)&p->toep_grid, (size_t)nb * tg->Kprod * sizeof(float2)));
    p->device_bytes += (int64_t)nb * tg->Kprod * (int64_t)sizeof(float2);
    p->toep_cap = nb;
  }
  tg->stream = p->stream;
  int rc = launch_fft_forward(tg, x, p->toep_grid, nb, false, h);
  if (rc != NUFFT_OK) return set_error(p, rc, "%s", tg->err);
  k_mul_spectrum<<<nblocks(tg->Kprod * nb), kThreads, 0, p->stream>>>(p->toep_grid, p->toep_T, tg->Kprod, nb);
  NUFFT_CUDA_TRY(p, cudaGetLastError());
  rc = launch_fft_inverse(tg, p->toep_grid, out, nb, false, h);
  if (rc != NUFFT_OK) return set_error(p, rc, "%s", tg->err);
  return NUFFT_OK;
}

}  // namespace

int normal_op_hooked(nufft_plan_t* p, float2* x, float2* out, const CgHooks* h) {
  if (p->normal_op == 1 && p->toep_T) return toeplitz_apply(p, x, out, 1, h);
  return selfadjoint_hooked(p, x, out, h);
}

int normal_op_epi_blocks(nufft_plan_t* p, int64_t* blocks) {
  if (p->normal_op == 1 && p->toep_T) {
    const int rc = fft_inverse_last_blocks(p->toep_geom, blocks);
    return rc == NUFFT_OK ? rc : set_error(p, rc, "%s", p->toep_geom->err);
  }
  return fft_inverse_last_blocks(p, blocks);
}

int normal_op(nufft_plan_t* p, const float2* x, float2* out, int nb) {
  if (p->normal_op == 1 && p->toep_T) return toeplitz_apply(p, x, out, nb);
  return selfadjoint_batch_impl(p, nb, x, out);
}

}  // namespace nufft

using namespace nufft;

extern "C" int nufft_toeplitz_init(nufft_plan_t* p) {
  if (!p) return set_error(nullptr, NUFFT_EINVAL, "plan is NULL");
  if (p->toep_T) return NUFFT_OK;
  const int d = p->g.d;
  // embedding period P = 2N rounded up to a power of two (>= 16); the kernel
  // comes from a P-image plan on a 2P grid
  int N2[kMaxDim], K2[kMaxDim], K4[kMaxDim], Nn[kMaxDim], J[kMaxDim];
  for (int a = 0; a < d; ++a) {
    int P = kMinK;
    while (P < 2 * p->g.N[a]) P *= 2;
    Nn[a] = p->g.N[a];
    N2[a] = K2[a] = P;
    K4[a] = 2 * P;
    J[a] = p->g.J[a];
    if (K4[a] > kMaxK)
      return set_error(p, NUFFT_EINVAL, "Toeplitz embedding needs a period P >= 2N with 2P <= %d (N[%d] = %d)",
                       kMaxK, a, p->g.N[a]);
  }
  cudaStream_t st = p->stream;
  // kernel t on the P image: adjoint NUFFT of all-ones with a P-image, 2P-grid plan
  DevBuf om_rows, ones, x2;
  PlanGuard big, full, geom;
  const int64_t M = p->M;
  if (M > 0) {
    NUFFT_CUDA_TRY(p, dev_malloc(&om_rows.ptr, M * d * sizeof(float)));
    k_om_rows<<<nblocks(M * d), kThreads, 0, st>>>(p->om_sorted, M, d, (float*)om_rows.ptr);
    NUFFT_CUDA_TRY(p, cudaGetLastError());
  }
  int rc = nufft_plan(d, N2, K4, J, M, (const float*)om_rows.ptr, st, &big.p);
  if (rc != NUFFT_OK) return set_error(p, rc, "Toeplitz kernel plan: %s", nufft_last_error(nullptr));
  int64_t n2 = 1;
  for (int a = 0; a < d; ++a) n2 *= N2[a];
  if (M > 0) {
    NUFFT_CUDA_TRY(p, dev_malloc(&ones.ptr, M * sizeof(float2)));
    k_fill<<<nblocks(M), kThreads, 0, st>>>((float2*)ones.ptr, M, make_float2(1.f, 0.f));
    NUFFT_CUDA_TRY(p, cudaGetLastError());
  }
  NUFFT_CUDA_TRY(p, dev_malloc(&x2.ptr, n2 * sizeof(float2)));
  rc = nufft_adjoint(big.p, (const float*)ones.ptr, (float*)x2.ptr);
  if (rc != NUFFT_OK) return set_error(p, rc, "Toeplitz kernel adjoint: %s", nufft_last_error(big.p));
  // T = DFT of the circular kernel.  A P image in a P grid is placed at
  // (n - P/2) mod P, which is exactly the circular arrangement t[D mod P].
  rc = nufft_plan(d, N2, K2, J, 0, nullptr, st, &full.p);
  if (rc != NUFFT_OK) return set_error(p, rc, "Toeplitz FFT plan: %s", nufft_last_error(nullptr));
  float2* T = nullptr;
  NUFFT_CUDA_TRY(p, dev_malloc((void**)&T, n2 * sizeof(float2)));
  rc = launch_fft_forward(full.p, (const float2*)x2.ptr, T, 1, false);
  if (rc != NUFFT_OK) {
    dev_free(T);
    return set_error(p, rc, "%s", full.p->err);
  }
  k_scale<<<nblocks(n2), kThreads, 0, st>>>(T, n2, (float)(1.0 / (double)n2));   // normalised inverse DFT
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    dev_free(T);
    return cuda_check(p, e, "Toeplitz kernel scale");
  }
  rc = nufft_plan(d, Nn, K2, J, 0, nullptr, st, &geom.p);
  if (rc != NUFFT_OK) {
    dev_free(T);
    return set_error(p, rc, "Toeplitz geometry plan: %s", nufft_last_error(nullptr));
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    dev_free(T);
    return cuda_check(p, e, "Toeplitz kernel");
  }
  p->toep_T = T;
  p->toep_geom = geom.p;
  geom.p = nullptr;
  p->device_bytes += n2 * (int64_t)sizeof(float2);
  return NUFFT_OK;
}

extern "C" int nufft_selfadjoint_toeplitz(nufft_plan_t* p, const float* x_dev, float* out_dev) {
  if (!p) return set_error(nullptr, NUFFT_EINVAL, "plan is NULL");
  if (!p->toep_T) return set_error(p, NUFFT_EINVAL, "call nufft_toeplitz_init first");
  if (!x_dev || !out_dev) return set_error(p, NUFFT_EINVAL, "x_dev or out_dev is NULL");
  return toeplitz_apply(p, reinterpret_cast<const float2*>(x_dev), reinterpret_cast<float2*>(out_dev), 1);
}

extern "C" int nufft_set_normal_operator(nufft_plan_t* p, int mode) {
  if (!p) return set_error(nullptr, NUFFT_EINVAL, "plan is NULL");
  if (mode != 0 && mode != 1) return set_error(p, NUFFT_EINVAL, "mode must be 0 (V^H V) or 1 (Toeplitz)");
  if (mode == 1 && !p->toep_T) return set_error(p, NUFFT_EINVAL, "call nufft_toeplitz_init first");
  if (mode != p->normal_op) drop_graphs(p);   // recorded solver graphs used the other operator
  p->normal_op = mode;
  return NUFFT_OK;
}
