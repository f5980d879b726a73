// fft.cu - scaling + zero-padding + oversampled FFT, and inverse FFT + crop +
// rescaling, as pruned line passes over the K^d grid.
//
// Section 2.1.1 (scaling S), Section 2.1.2 (zero-padding and oversampled FFT
// F; the inverse FFT followed by the array copy back), Table 1 rows S, F, F^H,
// S^H.  The paper runs S, a pre-indexed copy and a library FFT as separate
// steps over the whole K^d array.  Here the d-dimensional transform is done
// one axis at a time, and each pass is pruned:
//   forward, axis a: lines whose coordinates on axes < a lie in the padded
//     image's footprint (N_i of the K_i positions), all K on axes > a; only
//     the N_a non-zero inputs of a line are read; all K_a outputs written.
//     The first pass (last axis) reads the image itself and applies S, so
//     the padded array is never materialised.
//   inverse, axis a: lines over the crop footprint on axes < a, all K on
//     axes > a; all K_a inputs read, only the N_a cropped outputs written;
//     the last pass (last axis) applies S^H and writes the image.
// Padded position of image index n along an axis: g = (n - N/2) mod K.
//
// Each line of power-of-two length is transformed by a Stockham auto-sort
// FFT (one radix-2 or radix-4 stage, then radix-8 stages), each thread
// holding 8 values per stage in registers.  The first stage works on the values as loaded and
// the last stage's outputs are stored as they are; the hand-offs between
// stages go through two shared-memory buffers used in turn, one barrier per
// hand-off.  Twiddles exp(-2 pi i k / K) come from a table computed in FP64 at
// plan time and are loaded before the barrier of the stage that uses them.
// Other line lengths (even, prime factors 2, 3 and 5) run a Stockham FFT of
// radix-8, -4/-2, -3 and -5 stages through shared memory (k_fft_mixed).
#include "internal.cuh"

namespace nufft {
namespace {

struct FftArgs {
  const float2* src;
  float2* dst;
  const float* s_axis;        // scaling of axis a (image side only)
  const float* s_lead[kMaxDim];
  int a;
  int Na;                     // N_a
  int lead_N[kMaxDim];
  int lead_K[kMaxDim];
  int64_t lead_stride[kMaxDim];
  int64_t nouter;             // prod_{i<a} N_i
  int64_t inner;              // prod_{i>a} K_i (grid stride of axis a)
  int src_image;              // forward first pass: read the image, apply S
  int dst_image;              // inverse last pass: write the image, apply S^H
  int64_t src_bstride;        // batch strides (blockIdx.y selects the batch element)
  int64_t dst_bstride;
  int scale;                  // 0: no S / S^H (plain zero-pad / crop)
  // CG step hooks (see CgHooks): prologue of the first forward pass,
  // epilogue of the last inverse pass
  float2* pro_p;
  const float2* pro_r;
  const double* pro_part;
  int pro_count;
  double* pro_sc;
  int pro_old, pro_new;
  const float2* epi_a;
  double* epi_part;
};

// Sum of v over the CTA (any block size up to 1024) in a fixed order: a
// shuffle tree per warp, then the warps in order.  Every thread must call it;
// every thread gets the sum.  red: 32 doubles of shared scratch.
__device__ __forceinline__ double block_sum_dbl(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int w = 0; w < nw; ++w) t += red[w];
  __syncthreads();
  return t;
}

// beta of the CG prologue (every CTA computes the same value); CTA 0 stores
// the new <r, r> for the next step.
__device__ __forceinline__ float cg_prologue_beta(const FftArgs& A, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < A.pro_count; i += blockDim.x) s += A.pro_part[i];
  const double rr_new = block_sum_dbl(s, red);
  const double rr_old = A.pro_sc[A.pro_old];
  if (blockIdx.x == 0 && threadIdx.x == 0) A.pro_sc[A.pro_new] = rr_new;
  return (float)(rr_old != 0.0 ? rr_new / rr_old : 0.0);
}

// image element idx of the first forward pass: with the CG prologue,
// p = r + beta p written back in place (read with a plain load: it is written)
__device__ __forceinline__ float2 load_image(const FftArgs& A, const float2* __restrict__ src, int64_t idx,
                                             bool pro, float beta) {
  if (!pro) return __ldg(&src[idx]);
  const float2 pv = A.pro_p[idx], rv = A.pro_r[idx];
  const float2 pn = make_float2(fmaf(beta, pv.x, rv.x), fmaf(beta, pv.y, rv.y));
  A.pro_p[idx] = pn;
  return pn;
}

template <bool INV>
__device__ __forceinline__ float2 rot90(float2 z) {  // z * (-i) forward, z * (+i) inverse
  return INV ? make_float2(-z.y, z.x) : make_float2(z.y, -z.x);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2* v) {
  float2 a = v[0];
  v[0] = cadd(a, v[1]);
  v[1] = csub(a, v[1]);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& v0, float2& v1, float2& v2, float2& v3) {
  float2 a = cadd(v0, v2), b = csub(v0, v2), c = cadd(v1, v3), e = rot90<INV>(csub(v1, v3));
  v0 = cadd(a, c);
  v1 = cadd(b, e);
  v2 = csub(a, c);
  v3 = csub(b, e);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  const float h = 0.70710678118654752440f;
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  // o_k *= W8^k, W8 = exp(-+ 2 pi i / 8)
  o1 = INV ? make_float2(h * (o1.x - o1.y), h * (o1.x + o1.y))
           : make_float2(h * (o1.x + o1.y), h * (o1.y - o1.x));
  o2 = rot90<INV>(o2);
  o3 = INV ? make_float2(h * (-o3.x - o3.y), h * (o3.x - o3.y))
           : make_float2(h * (o3.y - o3.x), h * (-o3.x - o3.y));
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v) {
  if (R == 2) dft2<INV>(v);
  else if (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else dft8<INV>(v);
}

constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

// Shared-memory position of element p of the line owned by lane-group b.
// Contiguous axis: one line after another, one pad word per 8 elements.
// Strided axis: W lines side by side (W consecutive grid columns), row pitch W+1.
template <int L, bool STRIDED>
struct SmemMap {
  int w;  // lines per CTA
  static constexpr int kLinePitch = L + L / 8;
  __device__ __forceinline__ int at(int b, int p) const {
    return STRIDED ? p * (w + 1) + b : b * kLinePitch + p + (p >> 3);
  }
  __host__ __device__ static size_t words(int w) { return STRIDED ? (size_t)L * (w + 1) : (size_t)w * kLinePitch; }
};

// Stockham stage of radix R over span Ns on the values a thread holds.
//
// In every stage a thread reads the elements t + k*TPL (k = 0..7) of its line:
// butterfly q (q < 8/R) takes inputs j + r*L/R with j = t + q*TPL, which is
// element t + (q + r*Q)*TPL.  So x[k] holds element t + k*TPL on entry, the
// first stage needs no shared memory, and the outputs of the last stage
// (Ns = L/R, written to j + r*Ns) are again elements t + k*TPL, stored straight
// to global memory.  Only the middle hand-offs go through shared memory.
template <int L, int R>
struct StageTw {                      // twiddles of one stage
  float2 w[8 / R][R];
};

// Twiddles of a radix-8 stage, computed: input r of the thread's butterfly
// gets w1^r, w1 = exp(-+ 2 pi i k / (Ns R)), from sincospif (2k / (Ns R) is
// exact: Ns R is a power of two) and products of depth at most three (a few
// ulp; a table rounded from FP64 would be 0.5 ulp).  The passes then issue no
// twiddle loads (the strided 3D passes are bound by the L1/shared pipe, the
// 2D ones by load latency).
template <int L, bool INV>
__device__ __forceinline__ void make_twiddles8(StageTw<L, 8>& T, int t, int Ns) {
  const float inv = 2.0f / (float)(Ns * 8);   // exact
  const int k = t & (Ns - 1);                  // radix 8: one butterfly per thread
  float sn, cs;
  sincospif((float)k * inv, &sn, &cs);
  const float2 w1 = make_float2(cs, INV ? sn : -sn);
  const float2 w2 = cmul(w1, w1), w4 = cmul(w2, w2);
  T.w[0][1] = w1;
  T.w[0][2] = w2;
  T.w[0][3] = cmul(w2, w1);
  T.w[0][4] = w4;
  T.w[0][5] = cmul(w4, w1);
  T.w[0][6] = cmul(w4, w2);
  T.w[0][7] = cmul(w4, T.w[0][3]);
}

template <int L, bool INV, int R, bool TW>
__device__ __forceinline__ void butterflies(float2 (&x)[8], const StageTw<L, R>& T) {
  constexpr int Q = 8 / R;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[q + r * Q];
    if (TW) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], T.w[q][r]);
    }
    dft<R, INV>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) x[q + r * Q] = v[r];
  }
}

// Write the outputs of a stage (radix R, span Ns) to their Stockham positions.
template <int L, bool STRIDED, int R>
__device__ __forceinline__ void write_stage(float2* sm, const SmemMap<L, STRIDED> SI, int b, int t, int Ns,
                                            const float2 (&x)[8]) {
  constexpr int TPL = L / 8;
  constexpr int Q = 8 / R;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = t + q * TPL;
    const int k = j & (Ns - 1);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) sm[SI.at(b, base + r * Ns)] = x[q + r * Q];
  }
}

template <int L, bool STRIDED>
__device__ __forceinline__ void read_own(const float2* sm, const SmemMap<L, STRIDED> SI, int b, int t,
                                         float2 (&x)[8]) {
  constexpr int TPL = L / 8;
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = sm[SI.at(b, t + k * TPL)];
}

template <int L, bool STRIDED, bool INV>
__global__ void __launch_bounds__(STRIDED ? L : 256)
k_fft_pass(const FftArgs A, const int W) {
  constexpr int TPL = L / 8;
  const SmemMap<L, STRIDED> SI{W};
  extern __shared__ float2 sm[];
  const int bufw = (int)SmemMap<L, STRIDED>::words(W);   // buffer c at sm + c * bufw

  const int tid = threadIdx.x;
  int b, t;
  int64_t o, in;
  if (STRIDED) {
    b = tid % W;
    t = tid / W;
    const int64_t nib = A.inner / W;
    o = blockIdx.x / nib;
    in = (blockIdx.x % nib) * W + b;
  } else {
    b = tid / TPL;
    t = tid % TPL;
    o = (int64_t)blockIdx.x * W + b;
    in = 0;
  }
  const bool live = o < A.nouter;
  const float2* __restrict__ src = A.src + (int64_t)blockIdx.y * A.src_bstride;
  float2* __restrict__ dst = A.dst + (int64_t)blockIdx.y * A.dst_bstride;

  // Outer coordinates: image index on axes < a, mapped to padded grid positions.
  int64_t goff = 0;
  float slead = 1.0f;
  if (live) {
    int64_t rem = o;
    for (int i = A.a - 1; i >= 0; --i) {
      const int n = (int)(rem % A.lead_N[i]);
      rem /= A.lead_N[i];
      const int gi = wrapk(n - A.lead_N[i] / 2 + A.lead_K[i], A.lead_K[i]);
      goff += (int64_t)gi * A.lead_stride[i];
      if (A.scale && (A.src_image || A.dst_image)) slead *= A.s_lead[i][n];
    }
  }
  const int half = A.Na >> 1;
  const int64_t stride = A.inner;
  __shared__ double red[32];
  const bool pro = !INV && A.src_image && A.pro_p;
  const float beta = pro ? cg_prologue_beta(A, red) : 0.f;
  const uint64_t pol = l2_evict_first_policy();   // a pass reads each input element once

  constexpr int LOG = ilog2(L);
  constexpr int R0 = 1 << (LOG % 3);
  constexpr int N8 = LOG / 3;
  // ---- load the thread's elements t + k*TPL (pruned on the forward side)
  float2 x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int p = t + k * TPL;
    float2 v = make_float2(0.f, 0.f);
    if (live) {
      if (!INV) {
        const bool in_image = (p < half) || (p >= L - half);
        if (in_image) {
          if (A.src_image) {
            const int n = p < half ? p + half : p - L + half;
            v = cscale(load_image(A, src, o * A.Na + n, pro, beta), (A.scale ? A.s_axis[n] : 1.0f) * slead);
          } else {
            v = ld_last_use(&src[goff + (int64_t)p * stride + in], pol);
          }
        }
      } else {
        v = ld_last_use(&src[goff + (int64_t)p * stride + in], pol);
      }
    }
    x[k] = v;
  }

  // ---- transform: an optional radix-2/4 stage, then radix-8 stages
  int Ns = 1;
  int cur = 0;
  if (R0 > 1) {
    StageTw<L, R0> none;
    butterflies<L, INV, R0, false>(x, none);
    write_stage<L, STRIDED, R0>(sm, SI, b, t, 1, x);
    Ns = R0;
  }
#pragma unroll
  for (int s = 0; s < N8; ++s) {
    StageTw<L, 8> T;
    const bool first = (R0 == 1 && s == 0);
    if (!first) {
      make_twiddles8<L, INV>(T, t, Ns);
      __syncthreads();
      read_own<L, STRIDED>(sm + cur * bufw, SI, b, t, x);
      butterflies<L, INV, 8, true>(x, T);
    } else {
      butterflies<L, INV, 8, false>(x, T);
    }
    if (s + 1 < N8) {
      const int nxt = first ? 0 : cur ^ 1;
      write_stage<L, STRIDED, 8>(sm + nxt * bufw, SI, b, t, Ns, x);
      cur = nxt;
    }
    Ns *= 8;
  }

  // ---- store the thread's elements t + k*TPL (pruned on the inverse side)
  const bool epi = INV && A.dst_image && A.epi_part;
  double dot = 0.0;
  if (live) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int p = t + k * TPL;
      const float2 v = x[k];
      if (!INV) {
        dst[goff + (int64_t)p * stride + in] = v;
      } else {
        const bool in_image = (p < half) || (p >= L - half);
        if (!in_image) continue;
        if (A.dst_image) {
          const int n = p < half ? p + half : p - L + half;
          const float2 out = cscale(v, (A.scale ? A.s_axis[n] : 1.0f) * slead);
          dst[o * A.Na + n] = out;
          if (epi) {
            const float2 a = A.epi_a[o * A.Na + n];
            dot += (double)a.x * (double)out.x + (double)a.y * (double)out.y;
          }
        } else {
          dst[goff + (int64_t)p * stride + in] = v;
        }
      }
    }
  }
  if (epi) {
    const double tsum = block_sum_dbl(dot, red);
    if (threadIdx.x == 0) A.epi_part[blockIdx.x] = tsum;
  }
}

// Lines per CTA: as many as give 256 threads (8 columns on a strided axis, for
// 64-byte row segments), fewer when that would leave the GPU with fewer than
// two CTAs per SM (counting every batch element's CTAs).
constexpr int64_t kTargetBlocks = 2 * 152;

// query: only report the number of CTAs (per batch element) in *nblocks.
template <int L, bool STRIDED, bool INV>
cudaError_t launch_L(const FftArgs& A, int nb, cudaStream_t st, int64_t* nblocks, bool query) {
  constexpr int TPL = L / 8;
  int W;
  int64_t blocks;
  if (STRIDED) {
    W = 8;
    while (W > 2 && (A.inner % W != 0 || A.nouter * (A.inner / W) * nb < kTargetBlocks ||
                     2 * SmemMap<L, STRIDED>::words(W) * sizeof(float2) > 96 * 1024))
      W >>= 1;
    blocks = A.nouter * (A.inner / W);
  } else {
    W = TPL >= 256 ? 1 : 256 / TPL;
    while (W > 1 && (A.nouter + W - 1) / W * nb < kTargetBlocks) W >>= 1;
    blocks = (A.nouter + W - 1) / W;
  }
  if (nblocks) *nblocks = blocks;
  if (query) return cudaSuccess;
  const int threads = W * TPL;
  const size_t smem = 2 * SmemMap<L, STRIDED>::words(W) * sizeof(float2);   // ping-pong buffers
  // always: the kernel's static shared memory (the CG hooks' scratch) comes on
  // top, so even a 48 KB request needs the opt-in
  cudaError_t e = cudaFuncSetAttribute(k_fft_pass<L, STRIDED, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if (blocks == 0) return cudaSuccess;
  k_fft_pass<L, STRIDED, INV><<<dim3((unsigned)blocks, (unsigned)nb), threads, smem, st>>>(A, W);
  return cudaGetLastError();
}


// ---------------------------------------------------------------- other line lengths
// Stockham FFT of a line of length L = 2^a 3^b 5^c through shared memory:
// radix-8 stages, one radix-4 or radix-2 stage, then radix-3 and radix-5
// stages.  Stage s of radix R and span Ns (the product of the earlier radices)
// takes butterfly j (0 <= j < L/R) from elements j + r L/R, multiplies input
// r by exp(-+ 2 pi i r k / (Ns R)), k = j mod Ns, transforms the R values and
// writes output r to (j - k) R + k + r Ns.  The line sits in shared memory
// (two buffers used in turn, one barrier per stage); loads and stores are
// pruned and scaled as in k_fft_pass.
constexpr int kMaxStages = 16;
struct MixedRadix {
  int L;
  int nst;
  int radix[kMaxStages];
};

MixedRadix mixed_radix(int L) {
  MixedRadix m;
  memset(&m, 0, sizeof(m));
  m.L = L;
  int a = 0, v = L;
  while (v % 2 == 0) { v /= 2; ++a; }
  for (int i = 0; i < a / 3; ++i) m.radix[m.nst++] = 8;
  if (a % 3 == 2) m.radix[m.nst++] = 4;
  if (a % 3 == 1) m.radix[m.nst++] = 2;
  while (v % 3 == 0) { v /= 3; m.radix[m.nst++] = 3; }
  while (v % 5 == 0) { v /= 5; m.radix[m.nst++] = 5; }
  if (v != 1) m.nst = -1;   // not a supported length
  return m;
}

// DFT of 3 points: with w = exp(-+ 2 pi i / 3), y1 = v0 + w v1 + w^2 v2 and
// y2 = v0 + w^2 v1 + w v2 split into (v0 - (v1 + v2) / 2) -+ i (sqrt 3 / 2)(v1 - v2).
template <bool INV>
__device__ __forceinline__ void dft3(float2* v) {
  const float h = 0.86602540378443864676f;   // sqrt(3) / 2
  const float2 t1 = cadd(v[1], v[2]);
  const float2 t2 = make_float2(v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y);
  const float2 t3 = rot90<INV>(cscale(csub(v[1], v[2]), h));
  v[0] = cadd(v[0], t1);
  v[1] = cadd(t2, t3);
  v[2] = csub(t2, t3);
}

// DFT of 5 points: with c_k = cos(2 pi k / 5), s_k = sin(2 pi k / 5),
// y1, y4 = v0 + c1 (v1 + v4) + c2 (v2 + v3) -+ i (s1 (v1 - v4) + s2 (v2 - v3)),
// y2, y3 = v0 + c2 (v1 + v4) + c1 (v2 + v3) -+ i (s2 (v1 - v4) - s1 (v2 - v3)).
template <bool INV>
__device__ __forceinline__ void dft5(float2* v) {
  const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
  const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
  const float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  const float2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
  const float2 a1 = make_float2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
  const float2 a2 = make_float2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
  const float2 b1 = rot90<INV>(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
  const float2 b2 = rot90<INV>(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
  v[0] = make_float2(v[0].x + t1.x + t2.x, v[0].y + t1.y + t2.y);
  v[1] = cadd(a1, b1);
  v[4] = csub(a1, b1);
  v[2] = cadd(a2, b2);
  v[3] = csub(a2, b2);
}

template <bool STRIDED>
struct MixedMap {
  int w, L;   // lines per CTA, line length
  __device__ __forceinline__ int at(int b, int p) const { return STRIDED ? p * (w + 1) + b : b * (L + 1) + p; }
  __host__ __device__ static size_t words(int w, int L) { return (size_t)(STRIDED ? L * (w + 1) : w * (L + 1)); }
};

template <int R, bool INV, bool STRIDED>
__device__ __forceinline__ void mixed_stage(const float2* __restrict__ src, float2* __restrict__ dst,
                                            const MixedMap<STRIDED> SI, int b, int t, int TPL, int Ns) {
  const int L = SI.L;
  const int nbf = L / R;
  const float inv = 2.0f / (float)(Ns * R);
  for (int j = t; j < nbf; j += TPL) {
    const int k = j % Ns;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[SI.at(b, j + r * nbf)];
    if (Ns > 1) {   // input r times w1^r, w1 = exp(-+ 2 pi i k / (Ns R)), computed (no table loads)
      float sn, cs;
      sincospif((float)k * inv, &sn, &cs);
      const float2 w1 = make_float2(cs, INV ? sn : -sn);
      float2 w = w1;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        v[r] = cmul(v[r], w);
        if (r + 1 < R) w = cmul(w, w1);
      }
    }
    if (R == 3) dft3<INV>(v);
    else if (R == 5) dft5<INV>(v);
    else dft<R, INV>(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[SI.at(b, base + r * Ns)] = v[r];
  }
}

template <bool STRIDED, bool INV>
__global__ void __launch_bounds__(256)
k_fft_mixed(const FftArgs A, const int W, const __grid_constant__ MixedRadix mr) {
  const int L = mr.L;
  const int TPL = blockDim.x / W;
  const MixedMap<STRIDED> SI{W, L};
  extern __shared__ float2 sm[];
  const int bufw = (int)MixedMap<STRIDED>::words(W, L);

  const int tid = threadIdx.x;
  int b, t;
  int64_t o, in;
  if (STRIDED) {
    b = tid % W;
    t = tid / W;
    const int64_t nib = A.inner / W;
    o = blockIdx.x / nib;
    in = (blockIdx.x % nib) * W + b;
  } else {
    b = tid / TPL;
    t = tid % TPL;
    o = (int64_t)blockIdx.x * W + b;
    in = 0;
  }
  const bool live = o < A.nouter;
  const float2* __restrict__ src = A.src + (int64_t)blockIdx.y * A.src_bstride;
  float2* __restrict__ dst = A.dst + (int64_t)blockIdx.y * A.dst_bstride;

  int64_t goff = 0;
  float slead = 1.0f;
  if (live) {
    int64_t rem = o;
    for (int i = A.a - 1; i >= 0; --i) {
      const int n = (int)(rem % A.lead_N[i]);
      rem /= A.lead_N[i];
      const int gi = wrapk(n - A.lead_N[i] / 2 + A.lead_K[i], A.lead_K[i]);
      goff += (int64_t)gi * A.lead_stride[i];
      if (A.scale && (A.src_image || A.dst_image)) slead *= A.s_lead[i][n];
    }
  }
  const int half = A.Na >> 1;
  const int64_t stride = A.inner;
  __shared__ double red[32];
  const bool pro = !INV && A.src_image && A.pro_p;
  const float beta = pro ? cg_prologue_beta(A, red) : 0.f;
  const uint64_t pol = l2_evict_first_policy();   // a pass reads each input element once

  for (int p = t; p < L; p += TPL) {
    float2 v = make_float2(0.f, 0.f);
    if (live) {
      if (!INV) {
        if ((p < half) || (p >= L - half)) {
          if (A.src_image) {
            const int n = p < half ? p + half : p - L + half;
            v = cscale(load_image(A, src, o * A.Na + n, pro, beta), (A.scale ? A.s_axis[n] : 1.0f) * slead);
          } else {
            v = ld_last_use(&src[goff + (int64_t)p * stride + in], pol);
          }
        }
      } else {
        v = ld_last_use(&src[goff + (int64_t)p * stride + in], pol);
      }
    }
    sm[SI.at(b, p)] = v;
  }
  __syncthreads();

  int cur = 0, Ns = 1;
  for (int s = 0; s < mr.nst; ++s) {
    const int R = mr.radix[s];
    const float2* in_buf = sm + cur * bufw;
    float2* out_buf = sm + (cur ^ 1) * bufw;
    switch (R) {
      case 2: mixed_stage<2, INV>(in_buf, out_buf, SI, b, t, TPL, Ns); break;
      case 3: mixed_stage<3, INV>(in_buf, out_buf, SI, b, t, TPL, Ns); break;
      case 4: mixed_stage<4, INV>(in_buf, out_buf, SI, b, t, TPL, Ns); break;
      case 5: mixed_stage<5, INV>(in_buf, out_buf, SI, b, t, TPL, Ns); break;
      default: mixed_stage<8, INV>(in_buf, out_buf, SI, b, t, TPL, Ns); break;
    }
    __syncthreads();
    cur ^= 1;
    Ns *= R;
  }

  const float2* res = sm + cur * bufw;
  const bool epi = INV && A.dst_image && A.epi_part;
  double dot = 0.0;
  if (live) {
    for (int p = t; p < L; p += TPL) {
      const float2 v = res[SI.at(b, p)];
      if (!INV) {
        dst[goff + (int64_t)p * stride + in] = v;
      } else {
        if (!((p < half) || (p >= L - half))) continue;
        if (A.dst_image) {
          const int n = p < half ? p + half : p - L + half;
          const float2 out = cscale(v, (A.scale ? A.s_axis[n] : 1.0f) * slead);
          dst[o * A.Na + n] = out;
          if (epi) {
            const float2 a = A.epi_a[o * A.Na + n];
            dot += (double)a.x * (double)out.x + (double)a.y * (double)out.y;
          }
        } else {
          dst[goff + (int64_t)p * stride + in] = v;
        }
      }
    }
  }
  if (epi) {
    const double tsum = block_sum_dbl(dot, red);
    if (threadIdx.x == 0) A.epi_part[blockIdx.x] = tsum;
  }
}

// 256 threads per CTA: W lines of 256 / W threads (strided axes: W adjacent
// columns, W | inner), W lowered while the launch would give fewer than two
// CTAs per SM.
template <bool STRIDED, bool INV>
cudaError_t launch_mixed(int L, const FftArgs& A, int nb, cudaStream_t st, int64_t* nblocks, bool query) {
  const MixedRadix mr = mixed_radix(L);
  if (mr.nst < 0) return cudaErrorInvalidValue;
  int W;
  int64_t blocks;
  if (STRIDED) {
    W = 8;
    while (W > 1 && (A.inner % W != 0 || A.nouter * (A.inner / W) * nb < kTargetBlocks ||
                     2 * MixedMap<STRIDED>::words(W, L) * sizeof(float2) > 160 * 1024))
      W >>= 1;
    blocks = A.nouter * (A.inner / W);
  } else {
    const int tpl = L >= 512 ? 128 : (L >= 128 ? 64 : 32);
    W = 256 / tpl;
    while (W > 1 && (A.nouter + W - 1) / W * nb < kTargetBlocks) W >>= 1;
    blocks = (A.nouter + W - 1) / W;
  }
  if (nblocks) *nblocks = blocks;
  if (query) return cudaSuccess;
  const int threads = STRIDED ? 256 : W * (L >= 512 ? 128 : (L >= 128 ? 64 : 32));
  const size_t smem = 2 * MixedMap<STRIDED>::words(W, L) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_fft_mixed<STRIDED, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if (blocks == 0) return cudaSuccess;
  k_fft_mixed<STRIDED, INV><<<dim3((unsigned)blocks, (unsigned)nb), threads, smem, st>>>(A, W, mr);
  return cudaGetLastError();
}

template <bool STRIDED, bool INV>
cudaError_t launch_any(int L, const FftArgs& A, int nb, cudaStream_t st, int64_t* nblocks = nullptr,
                       bool query = false) {
  switch (L) {
    case 16: return launch_L<16, STRIDED, INV>(A, nb, st, nblocks, query);
    case 32: return launch_L<32, STRIDED, INV>(A, nb, st, nblocks, query);
    case 64: return launch_L<64, STRIDED, INV>(A, nb, st, nblocks, query);
    case 128: return launch_L<128, STRIDED, INV>(A, nb, st, nblocks, query);
    case 256: return launch_L<256, STRIDED, INV>(A, nb, st, nblocks, query);
    case 512: return launch_L<512, STRIDED, INV>(A, nb, st, nblocks, query);
    case 1024: return launch_L<1024, STRIDED, INV>(A, nb, st, nblocks, query);
    default: return launch_mixed<STRIDED, INV>(L, A, nb, st, nblocks, query);
  }
}

FftArgs make_args(const nufft_plan_t* p, int a) {
  FftArgs A;
  memset(&A, 0, sizeof(A));
  const Geom& g = p->g;
  A.a = a;
  A.Na = g.N[a];
  A.s_axis = p->s + p->s_off[a];
  A.nouter = 1;
  for (int i = 0; i < a; ++i) {
    A.lead_N[i] = g.N[i];
    A.lead_K[i] = g.K[i];
    A.lead_stride[i] = g.Kstride[i];
    A.s_lead[i] = p->s + p->s_off[i];
    A.nouter *= g.N[i];
  }
  A.inner = g.Kstride[a];
  return A;
}

}  // namespace

int launch_fft_forward(nufft_plan_t* p, const float2* x, float2* grid, int nb, bool scale, const CgHooks* h) {
  const int d = p->g.d;
  if (h && nb != 1) return set_error(p, NUFFT_EINVAL, "CG hooks need a single transform");
  for (int a = d - 1; a >= 0; --a) {
    FftArgs A = make_args(p, a);
    A.scale = scale ? 1 : 0;
    A.src_image = (a == d - 1);
    if (h && A.src_image && h->pro_p) {
      A.pro_p = h->pro_p;
      A.pro_r = h->pro_r;
      A.pro_part = h->pro_part;
      A.pro_count = h->pro_count;
      A.pro_sc = h->pro_sc;
      A.pro_old = h->pro_old;
      A.pro_new = h->pro_new;
    }
    A.src = A.src_image ? x : grid;
    A.dst = grid;
    A.src_bstride = A.src_image ? p->Nprod : p->Kprod;
    A.dst_bstride = p->Kprod;
    const bool strided = A.inner > 1;
    cudaError_t e = strided ? launch_any<true, false>(p->g.K[a], A, nb, p->stream)
                            : launch_any<false, false>(p->g.K[a], A, nb, p->stream);
    if (e != cudaSuccess) return cuda_check(p, e, "forward FFT pass");
  }
  return NUFFT_OK;
}

int fft_inverse_last_blocks(nufft_plan_t* p, int64_t* blocks) {
  const int a = p->g.d - 1;
  FftArgs A = make_args(p, a);
  A.dst_image = 1;
  const bool strided = A.inner > 1;
  cudaError_t e = strided ? launch_any<true, true>(p->g.K[a], A, 1, p->stream, blocks, true)
                          : launch_any<false, true>(p->g.K[a], A, 1, p->stream, blocks, true);
  return e == cudaSuccess ? NUFFT_OK : cuda_check(p, e, "inverse FFT pass");
}

int launch_fft_inverse(nufft_plan_t* p, float2* grid, float2* x, int nb, bool scale, const CgHooks* h) {
  const int d = p->g.d;
  if (h && nb != 1) return set_error(p, NUFFT_EINVAL, "CG hooks need a single transform");
  for (int a = 0; a < d; ++a) {
    FftArgs A = make_args(p, a);
    A.scale = scale ? 1 : 0;
    A.dst_image = (a == d - 1);
    A.src = grid;
    A.dst = A.dst_image ? x : grid;
    A.src_bstride = p->Kprod;
    A.dst_bstride = A.dst_image ? p->Nprod : p->Kprod;
    const bool epi = h && A.dst_image && h->epi_part;
    if (epi) {
      A.epi_a = h->epi_a;
      A.epi_part = h->epi_part;
    }
    const bool strided = A.inner > 1;
    int64_t blocks = 0;
    if (epi) {   // the block count first: the partial sums must fit
      cudaError_t e = strided ? launch_any<true, true>(p->g.K[a], A, nb, p->stream, &blocks, true)
                              : launch_any<false, true>(p->g.K[a], A, nb, p->stream, &blocks, true);
      if (e != cudaSuccess) return cuda_check(p, e, "inverse FFT pass");
      if (blocks > h->epi_cap)
        return set_error(p, NUFFT_EINVAL, "CG hooks: %lld partial sums exceed the capacity %d", (long long)blocks,
                         h->epi_cap);
      *h->epi_count = (int)blocks;
    }
    cudaError_t e = strided ? launch_any<true, true>(p->g.K[a], A, nb, p->stream)
                            : launch_any<false, true>(p->g.K[a], A, nb, p->stream);
    if (e != cudaSuccess) return cuda_check(p, e, "inverse FFT pass");
  }
  return NUFFT_OK;
}

}  // namespace nufft
