// plan.cu - plan creation: FP64 min-max interpolator precompute on the GPU,
// tile sort of the trajectory, work lists and plan-owned buffers.
//
// Section 2.1 (the min-max kernel of Fessler and Sutton is PyNUFFT's default)
// and Section 2.1.3 (the interpolator is precomputed once; the paper stores it
// as a CSR matrix).  Section 2.2.3 offloads its pre-indexes before the
// iterations start; the plan likewise does all index work once.
//
// Interpolator (one dimension; t_n = n - N/2, gamma = 2 pi / K):
//   s_n   = z_n / sinh(z_n), z_n = sqrt(alpha^2 - (pi J t_n / K)^2), alpha = 2.34 J
//           (sin for a negative radicand), normalised to max_n s_n = 1;
//   G     = [sum_n s_n^2 exp(i gamma (j - j') t_n)]_{j,j'=1..J},  T = G^{-1};
//   k0    = floor(w / gamma) - J/2 (J even), floor(w / gamma + 1/2) - (J+1)/2 (J odd);
//   r_j   = sum_n s_n exp(-i (w - gamma (k0 + j)) t_n),  c = T r.
// c minimises the worst-case interpolation error over unit-norm images (the
// least-squares solution of the min-max problem); the d-dimensional weight is
// the product of the per-dimension c.  All of it is computed in FP64 and the
// coefficients are stored as complex64.
#include <cmath>
#include <cstdarg>
#include <vector>

#include "internal.cuh"

namespace nufft {

static thread_local char g_err[512] = "no error";

int set_error(nufft_plan_t* p, int code, const char* fmt, ...) {
  char* dst = p ? p->err : g_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return code;
}

int cuda_check(nufft_plan_t* p, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return NUFFT_OK;
  if (e == cudaErrorMemoryAllocation)
    return set_error(p, NUFFT_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return set_error(p, NUFFT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

Points points_view(const nufft_plan_t* p) {
  Points P;
  P.M = p->M;
  P.kf = p->kf;
  P.coef = p->coef;
  for (int a = 0; a < kMaxDim; ++a) P.coef_off[a] = p->coef_off[a];
  P.perm = p->perm;
  P.cmax = p->cmax;
  return P;
}

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

// ---------------------------------------------------------------- per-dimension tables
struct DimTables {
  int d;
  int N[kMaxDim], K[kMaxDim], J[kMaxDim];
  int64_t s_off[kMaxDim];     // into s (float) and s64 (double)
  int64_t T_off[kMaxDim];     // into Tinv (double2), J*J each
};

__device__ double kb_recip_ft(double t, int J, int K) {
  const double alpha = 2.34 * J;
  const double q = alpha * alpha - (kPi * J * t / K) * (kPi * J * t / K);
  double ft;
  if (q > 0.0) {
    const double z = sqrt(q);
    ft = sinh(z) / z;
  } else if (q < 0.0) {
    const double z = sqrt(-q);
    ft = sin(z) / z;
  } else {
    ft = 1.0;
  }
  return 1.0 / ft;
}

// One CTA per dimension: scaling factors (max-normalised).
__global__ void k_scaling(DimTables D, float* s, double* s64) {
  const int a = blockIdx.x;
  const int N = D.N[a], K = D.K[a], J = D.J[a];
  __shared__ double red[256];
  double mx = 0.0;
  for (int n = threadIdx.x; n < N; n += blockDim.x) {
    const double v = kb_recip_ft((double)n - 0.5 * N, J, K);
    s64[D.s_off[a] + n] = v;
    mx = fmax(mx, v);
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  const double smax = red[0];
  for (int n = threadIdx.x; n < N; n += blockDim.x) {
    const double v = s64[D.s_off[a] + n] / smax;
    s64[D.s_off[a] + n] = v;
    s[D.s_off[a] + n] = (float)v;
  }
}

// One CTA per dimension: G (J x J, Hermitian) and its inverse by Gauss-Jordan
// elimination with partial pivoting, in FP64.
__global__ void k_minmax_T(DimTables D, const double* s64, double2* Tinv, int* singular) {
  const int a = blockIdx.x;
  const int N = D.N[a], K = D.K[a], J = D.J[a];
  const double gamma = 2.0 * kPi / K;
  __shared__ double2 Aug[kMaxJ][2 * kMaxJ];
  for (int e = threadIdx.x; e < J * J; e += blockDim.x) {
    const int r = e / J, c = e % J;
    double re = 0.0, im = 0.0;
    for (int n = 0; n < N; ++n) {
      const double sv = s64[D.s_off[a] + n];
      double sn, cs;
      sincos(gamma * (double)(r - c) * ((double)n - 0.5 * N), &sn, &cs);
      re += sv * sv * cs;
      im += sv * sv * sn;
    }
    Aug[r][c] = make_double2(re, im);
    Aug[r][J + c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int col = 0; col < J; ++col) {
      int piv = col;
      double best = -1.0;
      for (int r = col; r < J; ++r) {
        const double m = Aug[r][col].x * Aug[r][col].x + Aug[r][col].y * Aug[r][col].y;
        if (m > best) { best = m; piv = r; }
      }
      if (best <= 0.0) { *singular = 1; return; }
      if (piv != col)
        for (int c = 0; c < 2 * J; ++c) { double2 t = Aug[col][c]; Aug[col][c] = Aug[piv][c]; Aug[piv][c] = t; }
      // scale the pivot row by 1 / pivot
      const double2 pv = Aug[col][col];
      const double den = pv.x * pv.x + pv.y * pv.y;
      const double2 inv = make_double2(pv.x / den, -pv.y / den);
      for (int c = 0; c < 2 * J; ++c) {
        const double2 v = Aug[col][c];
        Aug[col][c] = make_double2(v.x * inv.x - v.y * inv.y, v.x * inv.y + v.y * inv.x);
      }
      for (int r = 0; r < J; ++r) {
        if (r == col) continue;
        const double2 f = Aug[r][col];
        for (int c = 0; c < 2 * J; ++c) {
          const double2 v = Aug[col][c];
          Aug[r][c].x -= f.x * v.x - f.y * v.y;
          Aug[r][c].y -= f.x * v.y + f.y * v.x;
        }
      }
    }
    for (int r = 0; r < J; ++r)
      for (int c = 0; c < J; ++c) Tinv[D.T_off[a] + r * J + c] = Aug[r][J + c];
  }
}

// floor-based first offset k0 (FP64), shared by the binning and coefficient kernels.
__device__ __forceinline__ double offset_k0(double w, int K, int J) {
  const double gamma = (2.0 * kPi) / K;
  const double u = w / gamma;
  return (J & 1) ? floor(u + 0.5) - (double)((J + 1) / 2) : floor(u) - (double)(J / 2);
}

__device__ __forceinline__ int wrap_first(double k0, int K) {
  // first neighbour k0 + 1, wrapped into [0, K)
  const long long k = (long long)k0 + 1;
  long long r = k % K;
  if (r < 0) r += K;
  return (int)r;
}

__global__ void k_validate(const float* om, int64_t n, int* bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = om[i];
    if (!(fabsf(v) <= 1048576.0f)) atomicOr(bad, 1);  // also catches NaN
  }
}

__global__ void k_bins(const float* om, int64_t M, Geom g, uint32_t* key, int32_t* val) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= M) return;
  uint32_t bin = 0;
  for (int a = 0; a < g.d; ++a) {
    const int kf = wrap_first(offset_k0((double)om[m * g.d + a], g.K[a], g.J[a]), g.K[a]);
    bin = bin * g.nb[a] + kf / g.T[a];
  }
  key[m] = bin;
  val[m] = (int32_t)m;
}

// ---------------------------------------------------------------- stable LSD radix sort (8 bits/pass)
constexpr int kSortThreads = 256;
constexpr int kSortItems = 4096;  // items per CTA

__global__ void k_radix_hist(const uint32_t* key, int64_t n, int shift, int nblk, uint32_t* hist) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t lo = (int64_t)blockIdx.x * kSortItems;
  const int64_t hi = min(n, lo + kSortItems);
  for (int64_t i = lo + threadIdx.x; i < hi; i += kSortThreads) atomicAdd(&h[(key[i] >> shift) & 255u], 1u);
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of n values with a single CTA of 1024 threads, in place
__global__ void k_scan_exclusive(uint32_t* v, int64_t n) {
  __shared__ uint32_t part[1024];
  const int64_t per = (n + 1023) / 1024;
  const int64_t lo = threadIdx.x * per;
  const int64_t hi = min(n, lo + per);
  uint32_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += v[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int t = 0; t < 1024; ++t) { const uint32_t c = part[t]; part[t] = run; run += c; }
  }
  __syncthreads();
  uint32_t run = part[threadIdx.x];
  for (int64_t i = lo; i < hi; ++i) { const uint32_t c = v[i]; v[i] = run; run += c; }
}

// Stable scatter: items of a CTA are ranked in their original order.
__global__ void k_radix_scatter(const uint32_t* kin, const int32_t* vin, uint32_t* kout, int32_t* vout,
                                int64_t n, int shift, int nblk, const uint32_t* offs) {
  __shared__ uint32_t running[256];
  __shared__ uint32_t wcount[kSortThreads / 32][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  running[tid] = offs[(int64_t)tid * nblk + blockIdx.x];
  const int64_t lo = (int64_t)blockIdx.x * kSortItems;
  for (int round = 0; round < kSortItems / kSortThreads; ++round) {
    for (int w = 0; w < kSortThreads / 32; ++w) wcount[w][tid] = 0;
    __syncthreads();
    const int64_t i = lo + (int64_t)round * kSortThreads + tid;
    const bool valid = i < n;
    const uint32_t k = valid ? kin[i] : 0u;
    const uint32_t digit = valid ? ((k >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    const unsigned lt = (1u << lane) - 1u;
    const int rank_w = __popc(peers & lt);
    if (valid && rank_w == 0) wcount[warp][digit] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t before = 0;
      for (int w = 0; w < warp; ++w) before += wcount[w][digit];
      const uint32_t pos = running[digit] + before + rank_w;
      kout[pos] = k;
      vout[pos] = vin[i];
    }
    __syncthreads();
    uint32_t tot = 0;
    for (int w = 0; w < kSortThreads / 32; ++w) tot += wcount[w][tid];
    running[tid] += tot;
    __syncthreads();
  }
}

// bin_start[b] = first sorted position with key >= b (binary search), b = 0..nbins
__global__ void k_bin_start(const uint32_t* key, int64_t M, int64_t nbins, int32_t* bin_start) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b > nbins) return;
  int64_t lo = 0, hi = M;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)key[mid] < b) lo = mid + 1; else hi = mid;
  }
  bin_start[b] = (int32_t)lo;
}

// The J min-max coefficients of one dimension (or, deriv = 1, their
// derivatives d c / d w with the neighbourhood fixed) for the offsets
// theta_j = w - gamma (k0 + j) = theta_1 - gamma (j - 1), j = 1..J:
//   r_j = sum_n s_n exp(-i theta_j t_n),  c = T r  (T = G^{-1}),
// and for the derivative the summand gains the factor -i t_n.  The sum runs
// with the rotation exp(-i theta) from its value at n = 0 (t = -N/2).
__device__ void minmax_coefs(double theta1, int N, int K, int J, const double* s, const double2* T, int deriv,
                             double2* c) {
  const double gamma = (2.0 * kPi) / K;
  double2 r[kMaxJ];
  for (int j = 1; j <= J; ++j) {
    const double theta = theta1 - gamma * (double)(j - 1);
    double sn, cs;
    sincos(-theta, &sn, &cs);            // rotation per step
    double es, ec;
    sincos(theta * 0.5 * N, &es, &ec);   // value at n = 0 (t = -N/2)
    double re = 0.0, im = 0.0;
    for (int n = 0; n < N; ++n) {
      if (deriv) {              // s_n (-i t_n) e_n = s_n t_n (es - i ec)
        const double st = s[n] * ((double)n - 0.5 * N);
        re += st * es;
        im -= st * ec;
      } else {
        re += s[n] * ec;
        im += s[n] * es;
      }
      const double nc = ec * cs - es * sn;
      const double ns = ec * sn + es * cs;
      ec = nc;
      es = ns;
    }
    r[j - 1] = make_double2(re, im);
  }
  for (int j = 0; j < J; ++j) {
    double re = 0.0, im = 0.0;
    for (int q = 0; q < J; ++q) {
      const double2 t = T[j * J + q];
      re += t.x * r[q].x - t.y * r[q].y;
      im += t.x * r[q].y + t.y * r[q].x;
    }
    c[j] = make_double2(re, im);
  }
}

// The coefficients depend on w only through the fractional offset
// delta = w / gamma - k0 - J/2 in [0, 1): theta_1 = gamma (delta + J/2 - 1).
// So per dimension they are smooth functions of one variable on [0, 1], and
// the plan expands each in Chebyshev polynomials of x = 2 delta - 1 (kCheb
// terms, coefficients from the values at the Chebyshev nodes), then evaluates
// the expansions per point (Clenshaw, FP64) instead of the N-term sums.  The
// expansion is checked against the sums at other points of [0, 1] and used
// only where it agrees to kChebTol relative to the largest coefficient.
constexpr int kCheb = 24;
constexpr double kChebTol = 1e-10;

__device__ __forceinline__ double cheb_node(int m) { return cos(kPi * (m + 0.5) / kCheb); }

// table layout: [(a * 2 + deriv) * kMaxJ + j] * kCheb + k
__global__ void k_cheb_fit(DimTables D, const double* s64, const double2* Tinv, double2* table) {
  const int a = blockIdx.x >> 1, deriv = blockIdx.x & 1;
  __shared__ double2 vals[kCheb][kMaxJ];
  const int N = D.N[a], K = D.K[a], J = D.J[a];
  const double gamma = (2.0 * kPi) / K;
  for (int m = threadIdx.x; m < kCheb; m += blockDim.x) {
    const double delta = 0.5 * (cheb_node(m) + 1.0);
    double2 c[kMaxJ];
    minmax_coefs(gamma * (delta + 0.5 * J - 1.0), N, K, J, s64 + D.s_off[a], Tinv + D.T_off[a], deriv, c);
    for (int j = 0; j < J; ++j) vals[m][j] = c[j];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < J * kCheb; t += blockDim.x) {
    const int j = t / kCheb, k = t - j * kCheb;
    double re = 0.0, im = 0.0;
    for (int m = 0; m < kCheb; ++m) {
      const double w = cos(kPi * k * (m + 0.5) / kCheb);
      re += w * vals[m][j].x;
      im += w * vals[m][j].y;
    }
    const double f = (k == 0 ? 1.0 : 2.0) / kCheb;
    table[((a * 2 + deriv) * kMaxJ + j) * kCheb + k] = make_double2(f * re, f * im);
  }
}

__device__ __forceinline__ double2 cheb_eval(const double2* a, double x) {
  double2 b1 = make_double2(0.0, 0.0), b2 = make_double2(0.0, 0.0);
  for (int k = kCheb - 1; k >= 1; --k) {
    const double2 b0 = make_double2(a[k].x + 2.0 * x * b1.x - b2.x, a[k].y + 2.0 * x * b1.y - b2.y);
    b2 = b1;
    b1 = b0;
  }
  return make_double2(a[0].x + x * b1.x - b2.x, a[0].y + x * b1.y - b2.y);
}

// Largest deviation of the expansion from the sums at kChebCheck points per
// (dimension, deriv), relative to the largest coefficient there; one block
// per (dimension, deriv), written to err[a * 2 + deriv].
constexpr int kChebCheck = 61;
__global__ void k_cheb_check(DimTables D, const double* s64, const double2* Tinv, const double2* table, double* err) {
  const int a = blockIdx.x >> 1, deriv = blockIdx.x & 1;
  const int N = D.N[a], K = D.K[a], J = D.J[a];
  const double gamma = (2.0 * kPi) / K;
  __shared__ double s_err[256], s_max[256];
  double e = 0.0, mx = 0.0;
  for (int t = threadIdx.x; t < kChebCheck; t += blockDim.x) {
    const double delta = (t + 0.5) / kChebCheck;
    double2 c[kMaxJ];
    minmax_coefs(gamma * (delta + 0.5 * J - 1.0), N, K, J, s64 + D.s_off[a], Tinv + D.T_off[a], deriv, c);
    for (int j = 0; j < J; ++j) {
      const double2 v = cheb_eval(table + ((a * 2 + deriv) * kMaxJ + j) * kCheb, 2.0 * delta - 1.0);
      e = fmax(e, hypot(v.x - c[j].x, v.y - c[j].y));
      mx = fmax(mx, hypot(c[j].x, c[j].y));
    }
  }
  s_err[threadIdx.x] = e;
  s_max[threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int t = 1; t < (int)blockDim.x; ++t) {
      e = fmax(e, s_err[t]);
      mx = fmax(mx, s_max[t]);
    }
    err[blockIdx.x] = mx > 0.0 ? e / mx : 0.0;
  }
}

// Per sorted point and dimension: first neighbour and the J min-max coefficients
// (deriv = 1: d c / d w instead).  cheb != NULL evaluates the plan's Chebyshev
// expansions, else the sums.  om_sorted = 1: om is [d][M] in sorted order;
// otherwise om is the caller's M x d array and perm maps to it, and the sorted
// copy is written to om_out (if not NULL).
__global__ void k_coefficients(const float* om, int om_sorted, Geom g, int64_t M, const int32_t* perm,
                               const double* s64, DimTables D, const double2* Tinv, int32_t* kf_out, float2* coef,
                               int64_t coef_off0, int64_t coef_off1, int64_t coef_off2, int deriv, float* om_out,
                               const double2* cheb) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= M * g.d) return;
  const int a = (int)(idx / M);
  const int64_t i = idx - (int64_t)a * M;
  const int N = g.N[a], K = g.K[a], J = g.J[a];
  const float wf = om_sorted ? om[(int64_t)a * M + i] : om[(int64_t)perm[i] * g.d + a];
  if (om_out) om_out[(int64_t)a * M + i] = wf;
  const double w = (double)wf;
  const double k0 = offset_k0(w, K, J);
  const double gamma = (2.0 * kPi) / K;
  const int64_t off = a == 0 ? coef_off0 : (a == 1 ? coef_off1 : coef_off2);
  if (cheb) {
    const double delta = w / gamma - k0 - 0.5 * J;
    const double x = fmin(1.0, fmax(-1.0, 2.0 * delta - 1.0));
    for (int j = 0; j < J; ++j) {
      const double2 v = cheb_eval(cheb + ((a * 2 + deriv) * kMaxJ + j) * kCheb, x);
      coef[off + (int64_t)j * M + i] = make_float2((float)v.x, (float)v.y);
    }
  } else {
    double2 c[kMaxJ];
    minmax_coefs(w - gamma * (k0 + 1.0), N, K, J, s64 + D.s_off[a], Tinv + D.T_off[a], deriv, c);
    for (int j = 0; j < J; ++j) coef[off + (int64_t)j * M + i] = make_float2((float)c[j].x, (float)c[j].y);
  }
  if (kf_out) kf_out[(int64_t)a * M + i] = wrap_first(k0, K);
}

// Largest coefficient magnitude of each dimension, as float bits (non-negative
// floats order like their bit patterns), for the gridding's fixed-point scale.
__global__ void k_coef_max(const float2* coef, int64_t M, int d, int J0, int J1, int J2, uint32_t* cmax) {
  const int64_t n0 = (int64_t)J0 * M, n1 = (int64_t)J1 * M, n2 = (int64_t)J2 * M;
  const int64_t n = n0 + (d > 1 ? n1 : 0) + (d > 2 ? n2 : 0);
  float m[kMaxDim] = {0.f, 0.f, 0.f};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 c = coef[i];
    const int a = i < n0 ? 0 : (i < n0 + n1 ? 1 : 2);
    m[a] = fmaxf(m[a], sqrtf(c.x * c.x + c.y * c.y));
  }
  for (int a = 0; a < d; ++a) {
    float v = m[a];
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&cmax[a], __float_as_uint(v));
  }
}

// Order each chunk's points for the gridding kernel.  Lane groups of J_last
// lanes handle one point each and G = 32 / J_last consecutive points share a
// warp instruction; point p's atomics for neighbour tap (j_0..j_{d-1}) land on
// the J_last consecutive shared-memory banks starting at
//   (cell index of its first neighbour in the padded tile + tap offset) mod 32,
// and the tap offset is the same for all points of an instruction.  So a
// group of G points whose first-neighbour windows [b, b + J_last) mod 32 are
// disjoint is free of bank conflicts for every one of its taps.  One thread
// per chunk buckets the points by b and forms the groups greedily, taking
// from the fullest bucket whose window is still free (a conflicting point
// only when no free window is left); stable and deterministic.
// One warp per chunk: the lanes compute the points' start banks b, lane k
// keeps bucket k (its count, and its points in chunk order in shared
// memory), and each greedy step is a warp-wide arg-max (fullest bucket whose
// window is free, lowest b on ties), so the order equals the one-thread
// greedy described above.  Shared memory per warp: b[cap] (bytes),
// ord[cap] and out[cap] (16-bit chunk positions), cap = chunk size (<= 2^15).
constexpr int kBankWarps = 4;

__global__ void __launch_bounds__(32 * kBankWarps)
k_bank_order(const float* om, Geom g, const Chunk* chunks, int64_t nchunks, const int32_t* perm_in,
             int32_t* perm_out, int cap) {
  extern __shared__ unsigned char sbank[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = blockIdx.x * (int64_t)kBankWarps + w;
  if (c >= nchunks) return;   // warp-uniform; only warp-level synchronisation below
  unsigned char* s_b = sbank + (size_t)w * cap * 5;
  int16_t* s_ord = reinterpret_cast<int16_t*>(s_b + cap);
  int16_t* s_out = s_ord + cap;
  const Chunk ch = chunks[c];
  const int d = g.d;
  const int JL = g.J[d - 1];
  const int G = 32 / JL;
  const unsigned base_mask = JL >= 32 ? 0xffffffffu : ((1u << JL) - 1u);
  int org[kMaxDim];
  {
    int rem = ch.bin;
    for (int a = d - 1; a >= 0; --a) {
      org[a] = (rem % g.nb[a]) * g.T[a];
      rem /= g.nb[a];
    }
  }
  for (int q = lane; q < ch.count; q += 32) {
    const int64_t m = perm_in[(int64_t)ch.start + q];
    int cell = 0;
    for (int a = 0; a < d; ++a) {
      const int kf = wrap_first(offset_k0((double)om[m * d + a], g.K[a], g.J[a]), g.K[a]);
      cell = cell * g.P[a] + (kf - org[a]);
    }
    s_b[q] = (unsigned char)(cell & 31);
  }
  __syncwarp();
  int cnt = 0;
  for (int q = 0; q < ch.count; ++q) cnt += s_b[q] == lane;
  int first = cnt;                                     // exclusive prefix over the lanes
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, first, o);
    if (lane >= o) first += v;
  }
  first -= cnt;
  for (int q = 0, pos = first; q < ch.count; ++q)
    if (s_b[q] == lane) s_ord[pos++] = (int16_t)q;
  __syncwarp();
  const unsigned my_win = (base_mask << lane) | (lane ? (base_mask >> (32 - lane)) : 0u);
  int head = first;
  int out = 0;
  while (out < ch.count) {
    unsigned used = 0u;
    for (int s = 0; s < G && out < ch.count; ++s) {
      // key: count + 1 in the high bits, 31 - lane low (ties -> lowest lane)
      const unsigned free_key = (cnt > 0 && (my_win & used) == 0u) ? ((unsigned)(cnt + 1) << 5) | (31u - lane) : 0u;
      unsigned best_key = __reduce_max_sync(0xffffffffu, free_key);
      if (best_key == 0u)
        best_key = __reduce_max_sync(0xffffffffu, cnt > 0 ? ((unsigned)(cnt + 1) << 5) | (31u - lane) : 0u);
      const int best = 31 - (int)(best_key & 31u);
      int q = 0;
      if (lane == best) {
        q = s_ord[head++];
        --cnt;
      }
      q = __shfl_sync(0xffffffffu, q, best);
      used |= (base_mask << best) | (best ? (base_mask >> (32 - best)) : 0u);
      if (lane == 0) s_out[out] = (int16_t)q;
      ++out;
    }
  }
  __syncwarp();
  for (int o = lane; o < ch.count; o += 32)
    perm_out[(int64_t)ch.start + o] = perm_in[(int64_t)ch.start + s_out[o]];
}

// K whose prime factors are all 2, 3 or 5 (the radices of the FFT passes).
bool fft_size_ok(int v) {
  if (v < 1) return false;
  for (int f : {2, 3, 5})
    while (v % f == 0) v /= f;
  return v == 1;
}

template <class T>
cudaError_t dalloc(nufft_plan_t* p, T** ptr, int64_t count) {
  *ptr = nullptr;
  if (count <= 0) return cudaSuccess;
  const size_t bytes = (size_t)count * sizeof(T);
  cudaError_t e = dev_malloc((void**)ptr, bytes);
  if (e == cudaSuccess) p->device_bytes += (int64_t)bytes;
  return e;
}

void free_plan_memory(nufft_plan_t* p) {
  void* bufs[] = {p->s, p->kf, p->coef, p->perm, p->bin_start, p->chunks, p->bin_chunk,
                  p->tiles, p->grid, p->ytmp, p->x_stage, p->y_stage, p->solver_ws, p->kspace_ws, p->mbuf,
                  p->s64, p->Tinv, p->om_sorted, p->dcoef, p->bgrid, p->btiles, p->bytmp, p->bimg,
                  p->cheb, p->sort_keys, p->sort_vals, p->sort_hist, p->perm2, p->flags, p->cmax, p->red_work};
  for (void* b : bufs)
    if (b) dev_free(b);
}

DimTables dim_tables(const nufft_plan_t* p) {
  DimTables D;
  memset(&D, 0, sizeof(D));
  D.d = p->g.d;
  for (int a = 0; a < p->g.d; ++a) {
    D.N[a] = p->g.N[a]; D.K[a] = p->g.K[a]; D.J[a] = p->g.J[a];
    D.s_off[a] = p->s_off[a]; D.T_off[a] = p->T_off[a];
  }
  return D;
}

int sort_blocks(int64_t M) { return (int)((M + kSortItems - 1) / kSortItems); }

// Reject a trajectory with a non-finite value or |om| > 2^20 (flag 0), before
// anything uses it.  Synchronizes the stream.
int validate_om(nufft_plan_t* p, const float* om) {
  cudaStream_t st = p->stream;
  NUFFT_CUDA_TRY(p, cudaMemsetAsync(p->flags, 0, sizeof(int), st));
  if (p->M > 0) {
    const int64_t n = p->M * p->g.d;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    k_validate<<<blocks, 256, 0, st>>>(om, n, p->flags);
    NUFFT_CUDA_TRY(p, cudaGetLastError());
  }
  int bad = 0;
  NUFFT_CUDA_TRY(p, cudaMemcpyAsync(&bad, p->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  NUFFT_CUDA_TRY(p, cudaStreamSynchronize(st));
  if (bad) return set_error(p, NUFFT_EINVAL, "om holds a non-finite value or |om| > 2^20");
  return NUFFT_OK;
}

// Everything that depends on the trajectory (validated already): the tile
// sort, the chunk list (chunks and partial tiles grown when it needs more),
// the bank order, the per-point interpolator and, once the trajectory
// gradient has been used, its derivative.  The per-dimension tables, the
// Chebyshev expansions and every other buffer are the plan's already.
int build_points(nufft_plan_t* p, const float* om) {
  Geom& g = p->g;
  const int d = g.d;
  const int64_t M = p->M;
  cudaStream_t st = p->stream;

  // ---- binning and stable sort by tile
  if (M > 0) {
    uint32_t* keyA = p->sort_keys;
    uint32_t* keyB = p->sort_keys + M;
    k_bins<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(om, M, g, keyA, p->perm);
    NUFFT_CUDA_TRY(p, cudaGetLastError());
    const int nblk = sort_blocks(M);
    int bits = 0;
    while ((int64_t(1) << bits) < g.nbins) ++bits;
    const int passes = std::max(1, (bits + 7) / 8);
    uint32_t* kin = keyA; uint32_t* kout = keyB;
    int32_t* vin = p->perm; int32_t* vout = p->sort_vals;
    for (int pass = 0; pass < passes; ++pass) {
      k_radix_hist<<<nblk, kSortThreads, 0, st>>>(kin, M, 8 * pass, nblk, p->sort_hist);
      k_scan_exclusive<<<1, 1024, 0, st>>>(p->sort_hist, (int64_t)256 * nblk);
      k_radix_scatter<<<nblk, kSortThreads, 0, st>>>(kin, vin, kout, vout, M, 8 * pass, nblk, p->sort_hist);
      NUFFT_CUDA_TRY(p, cudaGetLastError());
      std::swap(kin, kout);
      std::swap(vin, vout);
    }
    if (vin != p->perm)
      NUFFT_CUDA_TRY(p, cudaMemcpyAsync(p->perm, vin, M * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    k_bin_start<<<(unsigned)((g.nbins + 1 + 255) / 256), 256, 0, st>>>(kin, M, g.nbins, p->bin_start);
    NUFFT_CUDA_TRY(p, cudaGetLastError());
  } else {
    NUFFT_CUDA_TRY(p, cudaMemsetAsync(p->bin_start, 0, (g.nbins + 1) * sizeof(int32_t), st));
  }

  // ---- gridding work list: each tile's points cut into chunks
  std::vector<int32_t> bs(g.nbins + 1);
  NUFFT_CUDA_TRY(p, cudaMemcpyAsync(bs.data(), p->bin_start, (g.nbins + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                    st));
  NUFFT_CUDA_TRY(p, cudaStreamSynchronize(st));
  std::vector<Chunk> ch;
  std::vector<int32_t> bc(g.nbins + 1);
  for (int64_t b = 0; b < g.nbins; ++b) {
    bc[b] = (int32_t)ch.size();
    for (int32_t s0 = bs[b]; s0 < bs[b + 1]; s0 += kChunkPoints[d]) {
      Chunk c;
      c.bin = (int32_t)b;
      c.start = s0;
      c.count = std::min<int32_t>(kChunkPoints[d], bs[b + 1] - s0);
      c.pad = 0;
      ch.push_back(c);
    }
  }
  bc[g.nbins] = (int32_t)ch.size();
  const int64_t nch = (int64_t)ch.size();
  if (nch > p->chunk_cap) {   // grow the chunk list and the partial tiles (and the batched ones, lazily)
    drop_graphs(p);
    for (void* b : {(void*)p->chunks, (void*)p->tiles, (void*)p->btiles})
      if (b) dev_free(b);
    p->device_bytes -= p->chunk_cap * ((int64_t)sizeof(Chunk) + g.padded_cells * (int64_t)sizeof(float2)) +
                       (p->btiles ? (int64_t)p->batch_cap * p->chunk_cap * g.padded_cells * (int64_t)sizeof(float2) : 0);
    p->chunks = nullptr;
    p->tiles = nullptr;
    if (p->btiles) {   // the other batched buffers are re-made with it
      for (float2** b : {&p->bgrid, &p->bytmp, &p->bimg})
        if (*b) { dev_free(*b); *b = nullptr; }
      p->device_bytes -= (int64_t)p->batch_cap * (p->Kprod + M + p->Nprod) * (int64_t)sizeof(float2);
      p->btiles = nullptr;
      p->batch_cap = 0;
    }
    p->chunk_cap = 0;
    NUFFT_CUDA_TRY(p, dalloc(p, &p->chunks, nch));
    NUFFT_CUDA_TRY(p, dalloc(p, &p->tiles, nch * g.padded_cells));
    p->chunk_cap = nch;
  }
  p->nchunks = nch;
  if (nch > 0)
    NUFFT_CUDA_TRY(p, cudaMemcpyAsync(p->chunks, ch.data(), ch.size() * sizeof(Chunk), cudaMemcpyHostToDevice, st));
  NUFFT_CUDA_TRY(p, cudaMemcpyAsync(p->bin_chunk, bc.data(), bc.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                    st));

  // ---- 2D tile-reduction work list (single transforms): a dense tile (more
  // than 8 (neighbour, chunk) pairs, which its thread groups split) gets a CTA
  // of its own, {t, -2, -1, -1}; sparse tiles go NG to a CTA, one per group
  p->red_ctas = 0;
  if (d == 2 && nch > 0) {
    int gsize = 0, ng = 0;
    reduce2d_groups(g.T[0] * g.T[1], &gsize, &ng);
    if (gsize * ng <= 256) {
      const int nb0 = g.nb[0], nb1 = g.nb[1];
      std::vector<int4> wl;
      int pend[4] = {-1, -1, -1, -1}, fill = 0;
      for (int t = 0; t < (int)g.nbins; ++t) {
        const int b0 = t / nb1, b1 = t % nb1;
        int npairs = 0;
        for (int e = 0; e < 4; ++e) {
          const int src = ((b0 - (e >> 1) + nb0) % nb0) * nb1 + (b1 - (e & 1) + nb1) % nb1;
          npairs += bc[src + 1] - bc[src];
        }
        if (npairs > 8) {
          wl.push_back(make_int4(t, -2, -1, -1));
        } else {
          pend[fill++] = t;
          if (fill == ng) {
            wl.push_back(make_int4(pend[0], pend[1], pend[2], pend[3]));
            pend[0] = pend[1] = pend[2] = pend[3] = -1;
            fill = 0;
          }
        }
      }
      if (fill > 0) wl.push_back(make_int4(pend[0], pend[1], pend[2], pend[3]));
      if (!p->red_work) NUFFT_CUDA_TRY(p, dalloc(p, &p->red_work, g.nbins));
      NUFFT_CUDA_TRY(p, cudaMemcpyAsync(p->red_work, wl.data(), wl.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
      NUFFT_CUDA_TRY(p, cudaStreamSynchronize(st));   // wl is a host temporary
      p->red_ctas = (int)wl.size();
    }
  }

  // ---- order the points of each chunk for conflict-free shared-memory atomics
  if (M > 0 && nch > 0) {
    const int cap = kChunkPoints[d];
    static_assert(kChunkPoints[1] < 32768 && kChunkPoints[2] < 32768 && kChunkPoints[3] < 32768,
                  "16-bit chunk positions");
    const size_t smem = (size_t)kBankWarps * cap * 5;
    if (smem > 48 * 1024)
      NUFFT_CUDA_TRY(p, cudaFuncSetAttribute(k_bank_order, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_bank_order<<<(unsigned)((nch + kBankWarps - 1) / kBankWarps), 32 * kBankWarps, smem, st>>>(
        om, g, p->chunks, nch, p->perm, p->perm2, cap);
    NUFFT_CUDA_TRY(p, cudaGetLastError());
    NUFFT_CUDA_TRY(p, cudaMemcpyAsync(p->perm, p->perm2, M * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  }

  // ---- per-point interpolator in sorted order
  if (M > 0) {
    const DimTables D = dim_tables(p);
    const int64_t n = M * d;
    k_coefficients<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(om, 0, g, M, p->perm, p->s64, D, p->Tinv, p->kf,
                                                               p->coef, p->coef_off[0], p->coef_off[1],
                                                               p->coef_off[2], 0, p->om_sorted,
                                                               p->cheb_ok[0] ? p->cheb : nullptr);
    NUFFT_CUDA_TRY(p, cudaGetLastError());
    NUFFT_CUDA_TRY(p, cudaMemsetAsync(p->cmax, 0, kMaxDim * sizeof(uint32_t), st));
    k_coef_max<<<(unsigned)std::min<int64_t>(1024, (M * d + 255) / 256), 256, 0, st>>>(
        p->coef, M, d, g.J[0], d > 1 ? g.J[1] : 0, d > 2 ? g.J[2] : 0, p->cmax);
    NUFFT_CUDA_TRY(p, cudaGetLastError());
    if (p->dcoef) {
      k_coefficients<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(
          p->om_sorted, 1, g, M, p->perm, p->s64, D, p->Tinv, nullptr, p->dcoef, p->coef_off[0], p->coef_off[1],
          p->coef_off[2], 1, nullptr, p->cheb_ok[1] ? p->cheb : nullptr);
      NUFFT_CUDA_TRY(p, cudaGetLastError());
    }
  }
  return NUFFT_OK;
}

int build_plan(nufft_plan_t* p, const float* om) {
  Geom& g = p->g;
  const int d = g.d;
  const int64_t M = p->M;
  cudaStream_t st = p->stream;

  NUFFT_CUDA_TRY(p, dalloc(p, &p->flags, 2));
  NUFFT_CUDA_TRY(p, dalloc(p, &p->cmax, kMaxDim));
  NUFFT_CUDA_TRY(p, cudaMemsetAsync(p->cmax, 0, kMaxDim * sizeof(uint32_t), st));
  NUFFT_CUDA_TRY(p, cudaMemsetAsync(p->flags, 0, 2 * sizeof(int), st));
  int rc = validate_om(p, om);
  if (rc != NUFFT_OK) return rc;

  // ---- per-dimension tables
  int64_t s_tot = 0, T_tot = 0;
  for (int a = 0; a < d; ++a) {
    p->s_off[a] = s_tot; p->T_off[a] = T_tot;
    s_tot += g.N[a]; T_tot += (int64_t)g.J[a] * g.J[a];
  }
  const DimTables D = dim_tables(p);
  NUFFT_CUDA_TRY(p, dalloc(p, &p->s, s_tot));
  NUFFT_CUDA_TRY(p, dalloc(p, &p->s64, s_tot));
  NUFFT_CUDA_TRY(p, dalloc(p, &p->Tinv, T_tot));
  k_scaling<<<d, 256, 0, st>>>(D, p->s, p->s64);
  NUFFT_CUDA_TRY(p, cudaGetLastError());
  k_minmax_T<<<d, 256, 0, st>>>(D, p->s64, p->Tinv, p->flags + 1);
  NUFFT_CUDA_TRY(p, cudaGetLastError());

  // ---- Chebyshev expansions of the coefficients in the offset delta,
  // checked against the sums (kept for d c / d w too)
  int hflag[2] = {0, 0};
  if (M > 0) {
    NUFFT_CUDA_TRY(p, dalloc(p, &p->cheb, (int64_t)d * 2 * kMaxJ * kCheb));
    double* err = nullptr;
    NUFFT_CUDA_TRY(p, dev_malloc((void**)&err, 2 * kMaxDim * sizeof(double)));
    struct G5 { void* a; ~G5() { if (a) dev_free(a); } } g5{err};
    k_cheb_fit<<<2 * d, 64, 0, st>>>(D, p->s64, p->Tinv, p->cheb);
    NUFFT_CUDA_TRY(p, cudaGetLastError());
    k_cheb_check<<<2 * d, 64, 0, st>>>(D, p->s64, p->Tinv, p->cheb, err);
    NUFFT_CUDA_TRY(p, cudaGetLastError());
    double herr[2 * kMaxDim];
    NUFFT_CUDA_TRY(p, cudaMemcpyAsync(herr, err, 2 * d * sizeof(double), cudaMemcpyDeviceToHost, st));
    NUFFT_CUDA_TRY(p, cudaMemcpyAsync(hflag, p->flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    NUFFT_CUDA_TRY(p, cudaStreamSynchronize(st));
    p->cheb_ok[0] = p->cheb_ok[1] = 1;
    for (int a = 0; a < d; ++a)
      for (int v = 0; v < 2; ++v)
        if (!(herr[a * 2 + v] <= kChebTol)) p->cheb_ok[v] = 0;
  } else {
    NUFFT_CUDA_TRY(p, cudaMemcpyAsync(hflag, p->flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    NUFFT_CUDA_TRY(p, cudaStreamSynchronize(st));
  }
  if (hflag[1]) return set_error(p, NUFFT_EINVAL, "min-max matrix G is singular for these sizes");

  // ---- per-point arrays, sort scratch and work space
  int64_t coef_tot = 0;
  for (int a = 0; a < d; ++a) { p->coef_off[a] = coef_tot; coef_tot += (int64_t)g.J[a] * M; }
  NUFFT_CUDA_TRY(p, dalloc(p, &p->perm, M));
  NUFFT_CUDA_TRY(p, dalloc(p, &p->bin_start, g.nbins + 1));
  NUFFT_CUDA_TRY(p, dalloc(p, &p->bin_chunk, g.nbins + 1));
  NUFFT_CUDA_TRY(p, dalloc(p, &p->kf, M * d));
  NUFFT_CUDA_TRY(p, dalloc(p, &p->coef, coef_tot));
  NUFFT_CUDA_TRY(p, dalloc(p, &p->om_sorted, M * d));
  NUFFT_CUDA_TRY(p, dalloc(p, &p->sort_keys, 2 * M));
  NUFFT_CUDA_TRY(p, dalloc(p, &p->sort_vals, M));
  NUFFT_CUDA_TRY(p, dalloc(p, &p->sort_hist, M > 0 ? (int64_t)256 * sort_blocks(M) : 0));
  NUFFT_CUDA_TRY(p, dalloc(p, &p->perm2, M));
  rc = build_points(p, om);
  if (rc != NUFFT_OK) return rc;
  NUFFT_CUDA_TRY(p, dalloc(p, &p->grid, p->Kprod));
  NUFFT_CUDA_TRY(p, dalloc(p, &p->ytmp, M));
  NUFFT_CUDA_TRY(p, dalloc(p, &p->x_stage, p->Nprod));
  NUFFT_CUDA_TRY(p, dalloc(p, &p->y_stage, M));
  NUFFT_CUDA_TRY(p, cudaStreamSynchronize(st));
  return NUFFT_OK;
}

}  // namespace

int ensure_coef_derivatives(nufft_plan_t* p) {
  if (p->dcoef || p->M == 0) return NUFFT_OK;
  int64_t tot = 0;
  for (int a = 0; a < p->g.d; ++a) tot += (int64_t)p->g.J[a] * p->M;
  NUFFT_CUDA_TRY(p, dalloc(p, &p->dcoef, tot));
  DimTables D;
  memset(&D, 0, sizeof(D));
  D.d = p->g.d;
  for (int a = 0; a < p->g.d; ++a) {
    D.N[a] = p->g.N[a]; D.K[a] = p->g.K[a]; D.J[a] = p->g.J[a];
    D.s_off[a] = p->s_off[a]; D.T_off[a] = p->T_off[a];
  }
  const int64_t n = p->M * p->g.d;
  k_coefficients<<<(unsigned)((n + 127) / 128), 128, 0, p->stream>>>(
      p->om_sorted, 1, p->g, p->M, p->perm, p->s64, D, p->Tinv, nullptr, p->dcoef, p->coef_off[0], p->coef_off[1],
      p->coef_off[2], 1, nullptr, p->cheb_ok[1] ? p->cheb : nullptr);
  NUFFT_CUDA_TRY(p, cudaGetLastError());
  return NUFFT_OK;
}

}  // namespace nufft

using namespace nufft;

namespace {
int create_plan(int d, const int* Nd, const int* Kd, const int* Jd, int64_t M, const float* om_dev, void* stream,
                int tile_edge, nufft_plan_t** out) {
  if (!out) return set_error(nullptr, NUFFT_EINVAL, "out is NULL");
  *out = nullptr;
  if (d < 1 || d > kMaxDim) return set_error(nullptr, NUFFT_EINVAL, "d = %d, must be 1..3", d);
  if (!Nd || !Kd || !Jd) return set_error(nullptr, NUFFT_EINVAL, "Nd, Kd and Jd must not be NULL");
  if (M < 0 || M > 2147483647LL) return set_error(nullptr, NUFFT_EINVAL, "M = %lld out of range", (long long)M);
  if (M > 0 && !om_dev) return set_error(nullptr, NUFFT_EINVAL, "om_dev is NULL with M > 0");
  Geom g;
  memset(&g, 0, sizeof(g));
  g.d = d;
  const int base_tile = tile_edge > 0 ? tile_edge : (d == 1 ? 1024 : 16);
  for (int a = 0; a < d; ++a) {
    const int N = Nd[a], K = Kd[a], J = Jd[a];
    if ((K & 1) || !fft_size_ok(K) || K < kMinK || K > kMaxK)
      return set_error(nullptr, NUFFT_EINVAL,
                       "K[%d] = %d must be even, in [%d, %d], with no prime factor other than 2, 3 and 5", a, K,
                       kMinK, kMaxK);
    if (N < 2 || (N & 1) || N > K)
      return set_error(nullptr, NUFFT_EINVAL, "N[%d] = %d must be even with 2 <= N <= K = %d", a, N, K);
    if (J < 1 || J > kMaxJ || J > K)
      return set_error(nullptr, NUFFT_EINVAL, "J[%d] = %d must satisfy 1 <= J <= min(16, K)", a, J);
    g.N[a] = N; g.K[a] = K; g.J[a] = J;
    // tile edge: the largest divisor of K not above the base edge; if that is
    // below J - 1 (a point's footprint would reach past the next tile), the
    // smallest divisor of K from J - 1 up
    int T = 1;
    for (int t = std::min(base_tile, K); t >= 1; --t)
      if (K % t == 0) { T = t; break; }
    if (T < J - 1)
      for (int t = J - 1; t <= K; ++t)
        if (K % t == 0) { T = t; break; }
    g.T[a] = T;
    g.nb[a] = K / T;
    g.P[a] = T + J - 1;
  }
  int64_t stride = 1;
  g.nbins = 1;
  g.padded_cells = 1;
  for (int a = d - 1; a >= 0; --a) {
    g.Kstride[a] = stride;
    stride *= g.K[a];
    g.nbins *= g.nb[a];
    g.padded_cells *= g.P[a];
  }
  // the gridding accumulates a padded tile in shared memory: two 32-bit words
  // per cell (three in 3D)
  if (g.padded_cells * (int64_t)(d == 3 ? 12 : 8) > 200 * 1024)
    return set_error(nullptr, NUFFT_EINVAL, "padded gridding tile of %lld cells exceeds shared memory; lower J",
                     (long long)g.padded_cells);
  if (g.nbins > 65536) return set_error(nullptr, NUFFT_EINVAL, "too many tiles (%lld)", (long long)g.nbins);

  nufft_plan_t* p = new (std::nothrow) nufft_plan_t;
  if (!p) return set_error(nullptr, NUFFT_ENOMEM, "host allocation of the plan failed");
  memset(p, 0, sizeof(*p));
  p->g = g;
  p->M = M;
  p->Nprod = 1;
  p->Kprod = 1;
  for (int a = 0; a < d; ++a) { p->Nprod *= g.N[a]; p->Kprod *= g.K[a]; }
  p->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    cudaGetLastError();
    return set_error(nullptr, NUFFT_ECUDA, "cudaGetDevice failed");
  }
  p->graphs_enabled = 1;
  snprintf(p->err, sizeof(p->err), "no error");
  const int rc = build_plan(p, om_dev);
  if (rc != NUFFT_OK) {
    set_error(nullptr, rc, "%s", p->err);
    free_plan_memory(p);
    delete p;
    return rc;
  }
  *out = p;
  return NUFFT_OK;
}
}  // namespace

extern "C" int nufft_plan(int d, const int* Nd, const int* Kd, const int* Jd, int64_t M, const float* om_dev,
                          void* stream, nufft_plan_t** out) {
  return create_plan(d, Nd, Kd, Jd, M, om_dev, stream, 0, out);
}

// Tile-edge autotuner: one plan per candidate edge, each timed on a
// forward + adjoint pair (recorded graph, replayed kTuneReps times between
// CUDA events on the caller's stream); the fastest plan is returned and the
// others are destroyed.  Candidates: 1D 256/512/1024, 2D 8/16/32, 3D 8/16
// (each clipped to K; edges whose padded tile does not fit are skipped).
extern "C" int nufft_plan_tuned(int d, const int* Nd, const int* Kd, const int* Jd, int64_t M, const float* om_dev,
                                void* stream, nufft_plan_t** out) {
  if (!out) return set_error(nullptr, NUFFT_EINVAL, "out is NULL");
  *out = nullptr;
  if (d < 1 || d > kMaxDim) return set_error(nullptr, NUFFT_EINVAL, "d = %d, must be 1..3", d);
  const int cand1[] = {256, 512, 1024}, cand2[] = {8, 16, 32}, cand3[] = {8, 16};
  const int* cand = d == 1 ? cand1 : (d == 2 ? cand2 : cand3);
  const int ncand = d == 3 ? 2 : 3;
  constexpr int kTuneReps = 5;
  cudaStream_t st = (cudaStream_t)stream;
  nufft_plan_t* best = nullptr;
  float best_ms = 0.f;
  int last_rc = NUFFT_OK;
  float2 *xb = nullptr, *yb = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    if (xb) dev_free(xb);
    if (yb) dev_free(yb);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  for (int c = 0; c < ncand; ++c) {
    nufft_plan_t* p = nullptr;
    int rc = create_plan(d, Nd, Kd, Jd, M, om_dev, stream, cand[c], &p);
    if (rc != NUFFT_OK) {   // e.g. a padded tile too large for shared memory
      last_rc = rc;
      continue;
    }
    if (!xb) {
      cudaError_t e = dev_malloc((void**)&xb, p->Nprod * sizeof(float2));
      if (e == cudaSuccess && p->M > 0) e = dev_malloc((void**)&yb, p->M * sizeof(float2));
      if (e == cudaSuccess) e = cudaMemsetAsync(xb, 0, p->Nprod * sizeof(float2), st);
      if (e == cudaSuccess && yb) e = cudaMemsetAsync(yb, 0, p->M * sizeof(float2), st);
      if (e == cudaSuccess) e = cudaEventCreate(&e0);
      if (e == cudaSuccess) e = cudaEventCreate(&e1);
      if (e != cudaSuccess) {
        nufft_plan_destroy(p);
        if (best) nufft_plan_destroy(best);
        cleanup();
        cudaGetLastError();
        return set_error(nullptr, NUFFT_ECUDA, "autotune buffers: %s", cudaGetErrorString(e));
      }
    }
    float ms = 0.f;
    for (int it = 0; it < 2 + kTuneReps && rc == NUFFT_OK; ++it) {   // eager, record, then timed replays
      if (it == 2) rc = cuda_check(p, cudaEventRecord(e0, st), "autotune event");
      if (rc == NUFFT_OK) rc = nufft_forward(p, (const float*)xb, (float*)yb);
      if (rc == NUFFT_OK) rc = nufft_adjoint(p, (const float*)yb, (float*)xb);
    }
    if (rc == NUFFT_OK) rc = cuda_check(p, cudaEventRecord(e1, st), "autotune event");
    if (rc == NUFFT_OK) rc = cuda_check(p, cudaEventSynchronize(e1), "autotune event");
    if (rc == NUFFT_OK) rc = cuda_check(p, cudaEventElapsedTime(&ms, e0, e1), "autotune event");
    drop_graphs(p);   // the recorded graphs point at the scratch buffers
    if (rc != NUFFT_OK) {
      set_error(nullptr, rc, "%s", p->err);
      nufft_plan_destroy(p);
      if (best) nufft_plan_destroy(best);
      cleanup();
      return rc;
    }
    if (!best || ms < best_ms) {
      if (best) nufft_plan_destroy(best);
      best = p;
      best_ms = ms;
    } else {
      nufft_plan_destroy(p);
    }
  }
  cleanup();
  if (!best) return last_rc != NUFFT_OK ? last_rc : set_error(nullptr, NUFFT_EINVAL, "no tile edge fits");
  *out = best;
  return NUFFT_OK;
}

// Free the Toeplitz kernel, its work grid and its geometry plan.  The geometry
// plan is handed the owner's stream first: it last ran on whatever stream the
// owner used then (possibly the owner's capture stream, destroyed after this).
static void release_toeplitz(nufft_plan_t* p) {
  if (p->toep_geom) {
    p->toep_geom->stream = p->stream;
    nufft_plan_destroy(p->toep_geom);
    p->toep_geom = nullptr;
  }
  if (p->toep_T) dev_free(p->toep_T);
  if (p->toep_grid) dev_free(p->toep_grid);
  p->toep_T = nullptr;
  p->toep_grid = nullptr;
  p->toep_cap = 0;
}

extern "C" int nufft_plan_destroy(nufft_plan_t* p) {
  if (!p) return NUFFT_OK;
  cudaStreamSynchronize(p->stream);
  drop_graphs(p);
  release_toeplitz(p);   // before the capture stream, which its geometry plan may still name
  if (p->capture_stream) cudaStreamDestroy(p->capture_stream);
  free_plan_memory(p);
  delete p;
  return NUFFT_OK;
}

extern "C" const char* nufft_last_error(const nufft_plan_t* p) { return p ? p->err : g_err; }

extern "C" int nufft_plan_set_trajectory(nufft_plan_t* p, const float* om_dev) {
  if (!p) return set_error(nullptr, NUFFT_EINVAL, "plan is NULL");
  if (p->M > 0 && !om_dev) return set_error(p, NUFFT_EINVAL, "om_dev is NULL");
  int rc = validate_om(p, om_dev);   // the plan is unchanged when this fails
  if (rc != NUFFT_OK) return rc;
  drop_graphs(p);                    // recorded launches carry the old chunk count
  if (p->toep_T) {                   // the Toeplitz kernel belongs to the old trajectory
    release_toeplitz(p);
    p->normal_op = 0;
  }
  rc = build_points(p, om_dev);
  if (rc != NUFFT_OK) return rc;
  NUFFT_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
  return NUFFT_OK;
}

extern "C" int nufft_set_stream(nufft_plan_t* p, void* stream) {
  if (!p) return set_error(nullptr, NUFFT_EINVAL, "plan is NULL");
  p->stream = (cudaStream_t)stream;
  return NUFFT_OK;
}

extern "C" int nufft_plan_info(const nufft_plan_t* p, int64_t* info) {
  if (!p || !info) return set_error(nullptr, NUFFT_EINVAL, "plan or info is NULL");
  for (int i = 0; i < 16; ++i) info[i] = 0;
  info[0] = p->g.d;
  info[1] = p->M;
  for (int a = 0; a < p->g.d; ++a) {
    info[2 + a] = p->g.N[a];
    info[5 + a] = p->g.K[a];
    info[8 + a] = p->g.J[a];
  }
  info[11] = p->g.nbins;
  info[12] = p->nchunks;
  info[13] = p->device_bytes;
  info[14] = p->g.T[0];
  info[15] = p->g.T[p->g.d - 1];
  return NUFFT_OK;
}

extern "C" int nufft_plan_get_interpolator(const nufft_plan_t* cp, int32_t* kfirst_host, float* coef_host,
                                           float* s_host, int32_t* perm_host) {
  nufft_plan_t* p = const_cast<nufft_plan_t*>(cp);
  if (!p) return set_error(nullptr, NUFFT_EINVAL, "plan is NULL");
  const int d = p->g.d;
  const int64_t M = p->M;
  NUFFT_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
  std::vector<int32_t> perm(M), kf(M * d);
  if (M > 0) {
    NUFFT_CUDA_TRY(p, cudaMemcpy(perm.data(), p->perm, M * sizeof(int32_t), cudaMemcpyDeviceToHost));
    NUFFT_CUDA_TRY(p, cudaMemcpy(kf.data(), p->kf, M * d * sizeof(int32_t), cudaMemcpyDeviceToHost));
  }
  if (perm_host) for (int64_t i = 0; i < M; ++i) perm_host[i] = perm[i];
  if (kfirst_host)
    for (int a = 0; a < d; ++a)
      for (int64_t i = 0; i < M; ++i) kfirst_host[(int64_t)perm[i] * d + a] = kf[(int64_t)a * M + i];
  if (coef_host && M > 0) {
    int64_t out_off = 0;
    for (int a = 0; a < d; ++a) {
      const int J = p->g.J[a];
      std::vector<float2> c((size_t)J * M);
      NUFFT_CUDA_TRY(p, cudaMemcpy(c.data(), p->coef + p->coef_off[a], c.size() * sizeof(float2), cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < M; ++i)
        for (int j = 0; j < J; ++j) {
          const float2 v = c[(size_t)j * M + i];
          coef_host[out_off + ((int64_t)perm[i] * J + j) * 2] = v.x;
          coef_host[out_off + ((int64_t)perm[i] * J + j) * 2 + 1] = v.y;
        }
      out_off += (int64_t)2 * J * M;
    }
  }
  if (s_host) {
    int64_t off = 0;
    for (int a = 0; a < d; ++a) {
      NUFFT_CUDA_TRY(p, cudaMemcpy(s_host + off, p->s + p->s_off[a], p->g.N[a] * sizeof(float), cudaMemcpyDeviceToHost));
      off += p->g.N[a];
    }
  }
  return NUFFT_OK;
}
