// solvers.cu - CG, L1TV-OLS and L1TV-LAD on the NUFFT normal operator.
//
// The normal operator A^H A is applied through the grid (V^H V) or, after
// nufft_toeplitz_init and nufft_set_normal_operator(plan, 1), by its Toeplitz
// embedding.
// Section 2.1.5 (normal equation A^H A x = A^H y, Eq. 4), Section 2.2.2 (CG,
// Eqs. 7-9, both the image-domain form and the paper's own k-space form
// V^H V k = V^H y followed by x = S^{-1} F^{-1} k), Section 2.2.3 (image
// gradient by rolling, Eq. 10; L1TV-OLS, Eqs. 11-20; L1TV-LAD, Eqs. 21-31;
// multi-coil normal operator, Eqs. 32-33).  Bulk arithmetic is FP32; the inner
// products that set the CG step lengths are accumulated in FP64 in a fixed
// order (per-thread strided sums, a fixed shared-memory tree per CTA, then one
// CTA summing the per-CTA results), so a solve is reproducible for a given
// operator output.  Scalars stay in device memory: no host round trip per
// iteration.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace nufft {
int selfadjoint_impl(nufft_plan_t* p, const float2* x, float2* out);
int adjoint_dev(nufft_plan_t* p, const float2* y, float2* x);
int selfadjoint_multicoil_impl(nufft_plan_t* p, const float2* coils, int nc, const float2* x, float2* out);
int adjoint_multicoil_impl(nufft_plan_t* p, const float2* coils, int nc, const float2* y, float2* x);
}  // namespace nufft

using namespace nufft;

namespace {

constexpr int kDotBlocks = 304;      // 2 x 152 SMs: one 256-thread CTA per 256 elements of a 256^2 image
constexpr int kDotThreads = 256;
constexpr int kEwThreads = 256;

// scalar slots in device memory
enum { S_RR0 = 0, S_RR1 = 1, S_NSLOTS = 8 };

enum { V_B = 0, V_R, V_P, V_Q, V_AHY, V_AHYK, V_RHS, V_T, V_DF, V_BF, V_C1, V_C2, V_D0, V_B0 = V_D0 + 3,
       V_COUNT = V_B0 + 3 };

// partial sums of <p, A^H A p> written by the image-side inverse FFT pass of
// the fused CG (one per CTA of that pass)
constexpr int kEpiCap = 4096;

struct Ws {
  float2* v[V_COUNT];
  double* part;   // [2][kDotBlocks]: per-CTA partial sums (two sets in flight)
  double* sc;     // [S_NSLOTS]
  double* epi;    // [kEpiCap]
};

int get_ws(nufft_plan_t* p, Ws* w) {
  const int64_t n = p->Nprod;
  const int64_t vec_bytes = ((n * (int64_t)sizeof(float2) + 255) / 256) * 256;
  const int64_t bytes = vec_bytes * V_COUNT + (int64_t)(2 * kDotBlocks + S_NSLOTS + kEpiCap) * sizeof(double);
  if (!p->solver_ws) {
    cudaError_t e = dev_malloc(&p->solver_ws, bytes);
    if (e != cudaSuccess) { p->solver_ws = nullptr; return cuda_check(p, e, "solver work space"); }
    p->solver_ws_bytes = bytes;
    p->device_bytes += bytes;
  }
  char* base = (char*)p->solver_ws;
  for (int i = 0; i < V_COUNT; ++i) w->v[i] = (float2*)(base + vec_bytes * i);
  w->part = (double*)(base + vec_bytes * V_COUNT);
  w->sc = w->part + 2 * kDotBlocks;
  w->epi = w->sc + S_NSLOTS;
  return NUFFT_OK;
}

// --------------------------------------------------------------- reductions
__device__ __forceinline__ double block_sum(double v) {
  // a fixed shuffle tree in each warp, then the warps' sums in warp order;
  // every thread returns the same value
  __shared__ double red[kDotThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kDotThreads / 32; ++w) t += red[w];
  __syncthreads();   // red free for the next call
  return t;
}

// part[b] = sum over this CTA's strided share of Re(conj(a) b)
__global__ void __launch_bounds__(kDotThreads) k_dot_partial(const float2* a, const float2* b, int64_t n, double* part) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < n; i += (int64_t)kDotBlocks * kDotThreads) {
    const float2 u = a[i], v = b[i];
    s += (double)u.x * (double)v.x + (double)u.y * (double)v.y;
  }
  const double t = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kDotThreads) k_dot_final(const double* part, double* dst) {
  double s = 0.0;
  for (int i = threadIdx.x; i < kDotBlocks; i += kDotThreads) s += part[i];
  const double t = block_sum(s);
  if (threadIdx.x == 0) *dst = t;
}

// --------------------------------------------------------------- CG vector steps
__device__ __forceinline__ double safe_div(double a, double b) { return b != 0.0 ? a / b : 0.0; }

// Sum of the first `count` partial sums (kDotBlocks by default), in the same
// order in every CTA (so every CTA of a kernel gets the same value).
__device__ __forceinline__ double sum_partials(const double* part, int count = kDotBlocks) {
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += kDotThreads) s += part[i];
  return block_sum(s);
}

// x += alpha p, r -= alpha q, alpha = rr / <p, q> (<p, q> summed here from its
// partials); also the partial sums of <r, r>.
__global__ void __launch_bounds__(kDotThreads)
k_cg_xr(float2* x, float2* r, const float2* p, const float2* q, int64_t n, const double* sc, int rr_slot,
        const double* part_pq, int count_pq, double* part) {
  const float alpha = (float)safe_div(sc[rr_slot], sum_partials(part_pq, count_pq));
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < n; i += (int64_t)kDotBlocks * kDotThreads) {
    const float2 pv = p[i], qv = q[i];
    float2 xv = x[i], rv = r[i];
    xv.x = fmaf(alpha, pv.x, xv.x);
    xv.y = fmaf(alpha, pv.y, xv.y);
    rv.x = fmaf(-alpha, qv.x, rv.x);
    rv.y = fmaf(-alpha, qv.y, rv.y);
    x[i] = xv;
    r[i] = rv;
    s += (double)rv.x * (double)rv.x + (double)rv.y * (double)rv.y;
  }
  const double t = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// p = r + beta p, beta = rr_new / rr_old, rr_new summed here from its
// partials and kept in sc[new_slot] (by CTA 0) for the next step.
__global__ void __launch_bounds__(kDotThreads)
k_cg_p(float2* p, const float2* r, int64_t n, double* sc, int new_slot, int old_slot, const double* part_rr) {
  const double rr_new = sum_partials(part_rr);
  const float beta = (float)safe_div(rr_new, sc[old_slot]);
  if (blockIdx.x == 0 && threadIdx.x == 0) sc[new_slot] = rr_new;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 rv = r[i];
    float2 pv = p[i];
    pv.x = fmaf(beta, pv.x, rv.x);
    pv.y = fmaf(beta, pv.y, rv.y);
    p[i] = pv;
  }
}

// r = b - a, p = r (initial residual) with partial sums of <r, r>
__global__ void __launch_bounds__(kDotThreads)
k_cg_init(float2* r, float2* p, const float2* b, const float2* a, int64_t n, double* part) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < n; i += (int64_t)kDotBlocks * kDotThreads) {
    const float2 bv = b[i], av = a[i];
    const float2 rv = make_float2(bv.x - av.x, bv.y - av.y);
    r[i] = rv;
    p[i] = rv;
    s += (double)rv.x * (double)rv.x + (double)rv.y * (double)rv.y;
  }
  const double t = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// --------------------------------------------------------------- image-gradient kernels
struct ImgGeom {
  int d;
  int N[kMaxDim];
  int64_t stride[kMaxDim];
  int64_t n;
};

__device__ __forceinline__ int64_t nb_index(const ImgGeom& G, int64_t i, int a, int delta) {
  const int64_t c = (i / G.stride[a]) % G.N[a];
  int64_t c2 = c + delta;
  if (c2 < 0) c2 += G.N[a];
  if (c2 >= G.N[a]) c2 -= G.N[a];
  return i + (c2 - c) * G.stride[a];
}

// out = mu q + lambda sum_a (2 p - p[-e_a] - p[+e_a])   (K applied to p; q = A^H A p);
// part != NULL: also the CTA's partial sum of Re(conj(p) out) in part[blockIdx.x]
// (the CG step's <p, K p>; launched with kEwThreads == kDotThreads threads)
__global__ void __launch_bounds__(kEwThreads)
k_tv_apply(float2* out, const float2* q, const float2* p, ImgGeom G, float mu, float lam, double* part) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < G.n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 pv = p[i];
    float2 lap = make_float2(0.f, 0.f);
    for (int a = 0; a < G.d; ++a) {
      const float2 pm = p[nb_index(G, i, a, -1)], pp = p[nb_index(G, i, a, +1)];
      lap.x += 2.f * pv.x - pm.x - pp.x;
      lap.y += 2.f * pv.y - pm.y - pp.y;
    }
    const float2 qv = q[i];
    const float2 o = make_float2(mu * qv.x + lam * lap.x, mu * qv.y + lam * lap.y);
    out[i] = o;
    s += (double)pv.x * (double)o.x + (double)pv.y * (double)o.y;
  }
  if (part) {
    const double t = block_sum(s);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

// rhs = mu (base + df - bf) + lambda sum_a grad_a^T (d_a - b_a); df/bf may be NULL (OLS)
__global__ void k_rhs(float2* rhs, const float2* base, const float2* df, const float2* bf, const float2* d0,
                      const float2* b0, int64_t vstride, ImgGeom G, float mu, float lam) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < G.n; i += (int64_t)gridDim.x * blockDim.x) {
    float2 acc = base[i];
    if (df) {
      const float2 f = df[i], g = bf[i];
      acc.x += f.x - g.x;
      acc.y += f.y - g.y;
    }
    acc.x *= mu;
    acc.y *= mu;
    for (int a = 0; a < G.d; ++a) {
      const float2* da = d0 + a * vstride;
      const float2* ba = b0 + a * vstride;
      const int64_t im = nb_index(G, i, a, -1);
      // grad_a^T g [i] = g[i - e_a] - g[i]
      const float gx = (da[im].x - ba[im].x) - (da[i].x - ba[i].x);
      const float gy = (da[im].y - ba[im].y) - (da[i].y - ba[i].y);
      acc.x += lam * gx;
      acc.y += lam * gy;
    }
    rhs[i] = acc;
  }
}

__device__ __forceinline__ float2 shrink(float2 z, float t) {
  const float mag = sqrtf(z.x * z.x + z.y * z.y);
  if (mag == 0.f) return make_float2(0.f, 0.f);
  const float f = fmaxf(mag - t, 0.f) / mag;
  return make_float2(z.x * f, z.y * f);
}

// for every axis a: g = grad_a x; d_a = shrink(g + b_a, thr); b_a += g - d_a
__global__ void k_shrink_tv(const float2* x, float2* d0, float2* b0, int64_t vstride, ImgGeom G, float thr) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < G.n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 xv = x[i];
    for (int a = 0; a < G.d; ++a) {
      const float2 xp = x[nb_index(G, i, a, +1)];
      const float2 g = make_float2(xp.x - xv.x, xp.y - xv.y);
      float2* da = d0 + a * vstride;
      float2* ba = b0 + a * vstride;
      const float2 bv = ba[i];
      const float2 dv = shrink(make_float2(g.x + bv.x, g.y + bv.y), thr);
      da[i] = dv;
      ba[i] = make_float2(bv.x + (g.x - dv.x), bv.y + (g.y - dv.y));
    }
  }
}

// LAD data split: res = ahax - ahy; df = shrink(res + bf, thr); bf += res - df
__global__ void k_shrink_data(const float2* ahax, const float2* ahy, float2* df, float2* bf, int64_t n, float thr) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 a = ahax[i], h = ahy[i], bv = bf[i];
    const float2 res = make_float2(a.x - h.x, a.y - h.y);
    const float2 dv = shrink(make_float2(res.x + bv.x, res.y + bv.y), thr);
    df[i] = dv;
    bf[i] = make_float2(bv.x + (res.x - dv.x), bv.y + (res.y - dv.y));
  }
}

// Bregman outer step: ahyk += ahy - ahax
__global__ void k_outer(float2* ahyk, const float2* ahy, const float2* ahax, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 k = ahyk[i], h = ahy[i], a = ahax[i];
    ahyk[i] = make_float2(k.x + (h.x - a.x), k.y + (h.y - a.y));
  }
}

#define TRY(x)                       \
  do {                               \
    int _rc = (x);                   \
    if (_rc != NUFFT_OK) return _rc; \
  } while (0)
#define LAUNCH_CHECK(p, what) NUFFT_CUDA_TRY(p, cudaGetLastError())

// x[n] /= (K^d s[n]^2): turns S crop(F^H k) into S^{-1} crop(F^{-1} k)
__global__ void k_kspace_finish(float2* x, ImgGeom G, const float* s0, const float* s1, const float* s2,
                                float inv_kprod) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < G.n; i += (int64_t)gridDim.x * blockDim.x) {
    float sv = 1.f;
    const float* sp[3] = {s0, s1, s2};
    for (int a = 0; a < G.d; ++a) sv *= sp[a][(i / G.stride[a]) % G.N[a]];
    x[i] = cscale(x[i], inv_kprod / (sv * sv));
  }
}

int ew_blocks(int64_t n) {
  int64_t b = (n + kEwThreads - 1) / kEwThreads;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

ImgGeom img_geom(const nufft_plan_t* p) {
  ImgGeom G;
  memset(&G, 0, sizeof(G));
  G.d = p->g.d;
  int64_t s = 1;
  for (int a = G.d - 1; a >= 0; --a) {
    G.N[a] = p->g.N[a];
    G.stride[a] = s;
    s *= p->g.N[a];
  }
  G.n = s;
  return G;
}



// CG iterations on op x = b from the current x (in place), vectors of length n.
// r, pv, q are work vectors of length n; op(in, out) applies the operator.
template <class Op>
int cg_core(nufft_plan_t* p, int64_t n, float2* r, float2* pv, float2* q, double* part, double* sc, Op op,
            const float2* b, float2* x, int iters) {
  cudaStream_t st = p->stream;
  // part holds two sets of partial sums: <p, q> and <r, r>; the kernels that
  // need a full sum add the partials themselves (no separate final launch)
  double* part_pq = part;
  double* part_rr = part + kDotBlocks;
  TRY(op(x, q));
  k_cg_init<<<kDotBlocks, kDotThreads, 0, st>>>(r, pv, b, q, n, part_rr);
  k_dot_final<<<1, kDotThreads, 0, st>>>(part_rr, sc + S_RR0);
  LAUNCH_CHECK(p, "cg init");
  for (int it = 0; it < iters; ++it) {
    const int cur = (it & 1) ? S_RR1 : S_RR0;
    const int nxt = (it & 1) ? S_RR0 : S_RR1;
    TRY(op(pv, q));
    k_dot_partial<<<kDotBlocks, kDotThreads, 0, st>>>(pv, q, n, part_pq);
    k_cg_xr<<<kDotBlocks, kDotThreads, 0, st>>>(x, r, pv, q, n, sc, cur, part_pq, kDotBlocks, part_rr);
    k_cg_p<<<kDotBlocks, kDotThreads, 0, st>>>(pv, r, n, sc, nxt, cur, part_rr);
    LAUNCH_CHECK(p, "cg iteration");
  }
  return NUFFT_OK;
}

struct Operator {
  bool tv;       // false: A^H A; true: K = mu A^H A + lambda sum grad^T grad
  float mu, lam;
};

int apply_op(nufft_plan_t* p, const Operator& op, const float2* in, float2* out, float2* tmp) {
  if (!op.tv) return normal_op(p, in, out);
  TRY(normal_op(p, in, tmp));
  const ImgGeom G = img_geom(p);
  k_tv_apply<<<ew_blocks(G.n), kEwThreads, 0, p->stream>>>(out, tmp, in, G, op.mu, op.lam, nullptr);
  LAUNCH_CHECK(p, "tv apply");
  return NUFFT_OK;
}

// CG with the vector steps folded into the operator's kernels (see CgHooks):
// the forward FFT pass that reads p first applies the previous step's
// p = r + beta p, and the kernel that writes q = op(p) writes one partial sum
// of <p, q> per CTA (the image-side inverse FFT pass for A^H A, k_tv_apply for
// K = mu A^H A + lambda sum grad^T grad); one kernel per step remains (alpha,
// x += alpha p, r -= alpha q, partial <r, r>).  Seven launches per step for the
// 2D normal operator instead of nine; the same CG recurrence.
int cg_core_fused(nufft_plan_t* p, const Operator& op, int64_t n, float2* r, float2* pv, float2* q, float2* tmp,
                  double* part, double* sc, double* epi, const float2* b, float2* x, int iters) {
  cudaStream_t st = p->stream;
  double* part_rr = part + kDotBlocks;
  const ImgGeom G = img_geom(p);
  TRY(apply_op(p, op, x, q, tmp));
  k_cg_init<<<kDotBlocks, kDotThreads, 0, st>>>(r, pv, b, q, n, part_rr);
  k_dot_final<<<1, kDotThreads, 0, st>>>(part_rr, sc + S_RR0);
  LAUNCH_CHECK(p, "cg init");
  for (int it = 0; it < iters; ++it) {
    const int cur = (it & 1) ? S_RR1 : S_RR0;
    const int prev = (it & 1) ? S_RR0 : S_RR1;
    int count = 0;
    CgHooks h;
    if (it > 0) {   // the previous step's p update
      h.pro_p = pv;
      h.pro_r = r;
      h.pro_part = part_rr;
      h.pro_count = kDotBlocks;
      h.pro_sc = sc;
      h.pro_old = prev;
      h.pro_new = cur;
    }
    if (!op.tv) {
      h.epi_a = pv;
      h.epi_part = epi;
      h.epi_cap = kEpiCap;
      h.epi_count = &count;
      TRY(normal_op_hooked(p, pv, q, &h));
    } else {
      TRY(normal_op_hooked(p, pv, tmp, &h));
      count = ew_blocks(G.n);
      k_tv_apply<<<count, kEwThreads, 0, st>>>(q, tmp, pv, G, op.mu, op.lam, epi);
    }
    k_cg_xr<<<kDotBlocks, kDotThreads, 0, st>>>(x, r, pv, q, n, sc, cur, epi, count, part_rr);
    LAUNCH_CHECK(p, "cg iteration");
  }
  return NUFFT_OK;
}

// cg_iters CG steps on op x = b from the current x (in place), image-sized;
// the fused steps whenever the operator's partial sums fit kEpiCap.
int cg_run(nufft_plan_t* p, const Ws& w, const Operator& op, const float2* b, float2* x, int iters) {
  float2* t = w.v[V_T];
  int64_t epi_blocks = 0;
  if (op.tv) {
    epi_blocks = ew_blocks(p->Nprod);
  } else {
    TRY(normal_op_epi_blocks(p, &epi_blocks));
  }
  if (epi_blocks <= kEpiCap)
    return cg_core_fused(p, op, p->Nprod, w.v[V_R], w.v[V_P], w.v[V_Q], t, w.part, w.sc, w.epi, b, x, iters);
  return cg_core(p, p->Nprod, w.v[V_R], w.v[V_P], w.v[V_Q], w.part, w.sc,
                 [&](const float2* in, float2* out) { return apply_op(p, op, in, out, t); }, b, x, iters);
}

int check_common(nufft_plan_t* p, const float* y, const float* x) {
  if (!p) return set_error(nullptr, NUFFT_EINVAL, "plan is NULL");
  if (p->M > 0 && !y) return set_error(p, NUFFT_EINVAL, "y_dev is NULL");
  if (!x) return set_error(p, NUFFT_EINVAL, "x_dev is NULL");
  return NUFFT_OK;
}

int l1tv(nufft_plan_t* p, const float2* y, float2* x, int maxiter, int inner, int cg_iters, double mu, double lambda,
         bool lad) {
  Ws w;
  TRY(get_ws(p, &w));
  const int64_t n = p->Nprod;
  cudaStream_t st = p->stream;
  const ImgGeom G = img_geom(p);
  const int64_t vstride = w.v[1] - w.v[0];
  float2 *ahy = w.v[V_AHY], *ahyk = w.v[V_AHYK], *rhs = w.v[V_RHS], *tmp = w.v[V_B];
  float2 *df = w.v[V_DF], *bf = w.v[V_BF], *d0 = w.v[V_D0], *b0 = w.v[V_B0];
  TRY(adjoint_dev(p, y, ahy));
  NUFFT_CUDA_TRY(p, cudaMemcpyAsync(ahyk, ahy, n * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  for (int a = 0; a < G.d; ++a) {
    NUFFT_CUDA_TRY(p, cudaMemsetAsync(d0 + a * vstride, 0, n * sizeof(float2), st));
    NUFFT_CUDA_TRY(p, cudaMemsetAsync(b0 + a * vstride, 0, n * sizeof(float2), st));
  }
  if (lad) {
    NUFFT_CUDA_TRY(p, cudaMemsetAsync(df, 0, n * sizeof(float2), st));
    NUFFT_CUDA_TRY(p, cudaMemsetAsync(bf, 0, n * sizeof(float2), st));
  }
  const Operator K{true, (float)mu, (float)lambda};
  const float thr_tv = (float)(1.0 / lambda);
  const float thr_f = (float)(1.0 / mu);
  for (int outer = 0; outer < maxiter; ++outer) {
    for (int it = 0; it < inner; ++it) {
      k_rhs<<<ew_blocks(n), kEwThreads, 0, st>>>(rhs, ahyk, lad ? df : nullptr, lad ? bf : nullptr, d0, b0, vstride, G,
                                                (float)mu, (float)lambda);
      LAUNCH_CHECK(p, "rhs");
      TRY(cg_run(p, w, K, rhs, x, cg_iters));
      k_shrink_tv<<<ew_blocks(n), kEwThreads, 0, st>>>(x, d0, b0, vstride, G, thr_tv);
      LAUNCH_CHECK(p, "shrink");
      if (lad) {
        TRY(normal_op(p, x, tmp));
        k_shrink_data<<<ew_blocks(n), kEwThreads, 0, st>>>(tmp, ahy, df, bf, n, thr_f);
        LAUNCH_CHECK(p, "shrink data");
      }
    }
    // A^H A x of the last inner iteration: LAD already holds it in tmp (same x).
    if (!lad) TRY(normal_op(p, x, tmp));
    k_outer<<<ew_blocks(n), kEwThreads, 0, st>>>(ahyk, ahy, tmp, n);
    LAUNCH_CHECK(p, "outer");
  }
  return NUFFT_OK;
}

}  // namespace

extern "C" int solve_cg(nufft_plan_t* p, const float* y_dev, float* x_dev, int maxiter) {
  TRY(check_common(p, y_dev, x_dev));
  if (maxiter < 0) return set_error(p, NUFFT_EINVAL, "maxiter < 0");
  Ws w;
  TRY(get_ws(p, &w));
  const float2* y = reinterpret_cast<const float2*>(y_dev);
  float2* x = reinterpret_cast<float2*>(x_dev);
  return run_graphed(p, 7, y, x, maxiter, [&]() -> int {
    TRY(adjoint_dev(p, y, w.v[V_B]));
    const Operator op{false, 1.f, 0.f};
    return cg_run(p, w, op, w.v[V_B], x, maxiter);
  });
}

namespace {

int l1tv_entry(nufft_plan_t* p, const float* y_dev, float* x_dev, int maxiter, int inner, int cg_iters, double mu,
               double lambda, bool lad) {
  TRY(check_common(p, y_dev, x_dev));
  if (maxiter < 0 || inner < 1 || cg_iters < 1)
    return set_error(p, NUFFT_EINVAL, "need maxiter >= 0, inner >= 1, cg_iters >= 1");
  if (!(mu > 0.0) || !(lambda > 0.0)) return set_error(p, NUFFT_EINVAL, "need mu > 0 and lambda > 0");
  Ws w;
  TRY(get_ws(p, &w));
  const float2* y = reinterpret_cast<const float2*>(y_dev);
  float2* x = reinterpret_cast<float2*>(x_dev);
  return run_graphed(p, lad ? 9 : 8, y, x, graph_key({(uint64_t)maxiter, (uint64_t)inner, (uint64_t)cg_iters, graph_bits(mu), graph_bits(lambda)}),
                     [&]() { return l1tv(p, y, x, maxiter, inner, cg_iters, mu, lambda, lad); });
}

}  // namespace

extern "C" int solve_l1tv_ols(nufft_plan_t* p, const float* y_dev, float* x_dev, int maxiter, int inner,
                              int cg_iters, double mu, double lambda) {
  return l1tv_entry(p, y_dev, x_dev, maxiter, inner, cg_iters, mu, lambda, false);
}

extern "C" int solve_l1tv_lad(nufft_plan_t* p, const float* y_dev, float* x_dev, int maxiter, int inner,
                              int cg_iters, double mu, double lambda) {
  return l1tv_entry(p, y_dev, x_dev, maxiter, inner, cg_iters, mu, lambda, true);
}

// ------------------------------------------------------------------ k-space CG (Eqs. 7-9)
extern "C" int solve_cg_kspace(nufft_plan_t* p, const float* y_dev, float* x_dev, int maxiter) {
  TRY(check_common(p, y_dev, x_dev));
  if (maxiter < 0) return set_error(p, NUFFT_EINVAL, "maxiter < 0");
  Ws w;
  TRY(get_ws(p, &w));
  const int64_t n = p->Kprod;
  const int64_t vb = ((n * (int64_t)sizeof(float2) + 255) / 256) * 256;
  if (!p->kspace_ws) {
    cudaError_t e = dev_malloc(&p->kspace_ws, 5 * vb);
    if (e != cudaSuccess) { p->kspace_ws = nullptr; return cuda_check(p, e, "k-space CG work space"); }
    p->device_bytes += 5 * vb;
  }
  char* base = (char*)p->kspace_ws;
  float2 *b = (float2*)base, *r = (float2*)(base + vb), *pv = (float2*)(base + 2 * vb),
         *q = (float2*)(base + 3 * vb), *k = (float2*)(base + 4 * vb);
  return run_graphed(p, 10, y_dev, x_dev, maxiter, [&]() -> int {
    cudaStream_t st = p->stream;
    TRY(launch_gridding(p, reinterpret_cast<const float2*>(y_dev), b));          // V^H y
    NUFFT_CUDA_TRY(p, cudaMemsetAsync(k, 0, n * sizeof(float2), st));
    auto vhv = [&](const float2* in, float2* out) -> int {                       // V^H V
      if (vhv_fused(p)) return launch_vhv(p, in, out);
      TRY(launch_interp(p, in, p->ytmp));
      return launch_gridding(p, p->ytmp, out);
    };
    TRY(cg_core(p, n, r, pv, q, w.part, w.sc, vhv, b, k, maxiter));
    TRY(launch_fft_inverse(p, k, reinterpret_cast<float2*>(x_dev)));          // S crop(F^H k)
    const ImgGeom G = img_geom(p);
    const float* s1 = p->g.d > 1 ? p->s + p->s_off[1] : p->s;
    const float* s2 = p->g.d > 2 ? p->s + p->s_off[2] : p->s;
    k_kspace_finish<<<ew_blocks(G.n), kEwThreads, 0, st>>>(reinterpret_cast<float2*>(x_dev), G, p->s + p->s_off[0],
                                                          s1, s2, (float)(1.0 / (double)p->Kprod));
    LAUNCH_CHECK(p, "k-space finish");
    return NUFFT_OK;
  });
}

// ------------------------------------------------------------------ multi-coil CG (Eqs. 32-33)
extern "C" int solve_cg_multicoil(nufft_plan_t* p, const float* coils_dev, int nc, const float* y_dev, float* x_dev,
                                  int maxiter) {
  TRY(check_common(p, y_dev, x_dev));
  if (!coils_dev || nc < 1) return set_error(p, NUFFT_EINVAL, "coils_dev is NULL or nc < 1");
  if (maxiter < 0) return set_error(p, NUFFT_EINVAL, "maxiter < 0");
  Ws w;
  TRY(get_ws(p, &w));
  const float2* coils = reinterpret_cast<const float2*>(coils_dev);
  const float2* y = reinterpret_cast<const float2*>(y_dev);
  float2* x = reinterpret_cast<float2*>(x_dev);
  const int64_t key = graph_key({(uint64_t)maxiter, (uint64_t)nc, graph_bits(coils_dev)});
  return run_graphed(p, 15, y, x, key, [&]() -> int {
    TRY(adjoint_multicoil_impl(p, coils, nc, y, w.v[V_B]));
    auto op = [&](const float2* in, float2* out) -> int { return selfadjoint_multicoil_impl(p, coils, nc, in, out); };
    return cg_core(p, p->Nprod, w.v[V_R], w.v[V_P], w.v[V_Q], w.part, w.sc, op, w.v[V_B], x, maxiter);
  });
}
