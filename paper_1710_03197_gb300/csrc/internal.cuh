// internal.cuh - plan layout and kernel launchers shared by the library's
// translation units.  Not part of the public ABI (see include/nufft_gb300.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <initializer_list>

#include "../../include/nufft_gb300.h"

namespace nufft {

constexpr int kMaxDim = 3;
constexpr int kMaxJ = 16;
constexpr int kMinK = 16;
constexpr int kMaxK = 1024;
// Points per gridding chunk (by dimension): a tile's points are cut into
// chunks of at most this many so that a dense tile (the centre of a radial
// trajectory) is spread over several CTAs, and small problems still fill the
// GPU.  3D chunks are larger because each partial tile costs 74 KB.
constexpr int kChunkPoints[4] = {0, 1024, 256, 2048};

// Geometry of the oversampled grid and of the tile decomposition.
struct Geom {
  int d;
  int N[kMaxDim];      // image size
  int K[kMaxDim];      // grid size (even; prime factors 2, 3, 5)
  int J[kMaxDim];      // neighbours
  int T[kMaxDim];      // tile edge: a divisor of K with T >= J - 1
  int nb[kMaxDim];     // tiles per dimension = K / T
  int P[kMaxDim];      // padded tile edge = T + J - 1
  int64_t Kstride[kMaxDim];  // C-order strides of the grid
  int64_t nbins;
  int64_t padded_cells;      // prod P
};

// Per-point interpolator in tile-sorted order ("structure of arrays").
struct Points {
  int64_t M;
  const int32_t* kf;     // [d][M]  first neighbour, wrapped into [0, K)
  const float2* coef;    // dim i starts at coef + coef_off[i]; layout [J_i][M]
  int64_t coef_off[kMaxDim];
  const int32_t* perm;   // sorted position -> trajectory index
  const uint32_t* cmax;  // [d] largest |coefficient| of each dimension (float bits)
};

struct Chunk {
  int32_t bin;
  int32_t start;   // first sorted point
  int32_t count;   // points in this chunk
  int32_t pad;
};

}  // namespace nufft

namespace nufft {
// One cached executable graph of an entry point's launch sequence.
struct GraphEntry {
  int kind;                 // 0 = free slot
  const void* a;
  const void* b;
  int64_t extra;
  cudaStream_t stream;
  int state;                // 1: seen once (ran eagerly), 2: graph ready, 3: never graph
  cudaGraphExec_t exec;
  uint64_t last_use;
};
constexpr int kGraphSlots = 16;
}  // namespace nufft

struct nufft_plan {
  nufft::Geom g;
  int64_t M;
  int64_t Nprod;
  int64_t Kprod;
  cudaStream_t stream;
  int device;               // CUDA device current when the plan was made (its memory lives there)

  // plan-owned device memory
  float* s;                 // scaling, dim i at s + s_off[i]
  int64_t s_off[nufft::kMaxDim];
  int32_t* kf;              // [d][M] sorted
  float2* coef;             // [sum_i J_i][M] sorted
  int64_t coef_off[nufft::kMaxDim];
  int32_t* perm;            // [M]
  int32_t* bin_start;       // [nbins + 1]
  nufft::Chunk* chunks;     // [nchunks]
  int32_t* bin_chunk;       // [nbins + 1] chunk range of each bin
  int64_t nchunks;
  float2* tiles;            // [nchunks][padded_cells] gridding partial tiles
  float2* grid;             // [Kprod] oversampled grid work space
  float2* ytmp;             // [M] work space of the self-adjoint operator
  float2* x_stage;          // [Nprod] staging for host-buffer calls
  float2* y_stage;          // [M]
  int64_t device_bytes;

  // solver work space (allocated on first solver call)
  void* solver_ws;
  int64_t solver_ws_bytes;
  // k-space CG work space (grid-sized vectors) and an M-sized buffer,
  // allocated on first use by the calls that need them
  void* kspace_ws;
  float2* mbuf;

  // kept from plan creation for the trajectory derivative
  double* s64;              // scaling in FP64, dim i at s_off[i]
  double2* Tinv;            // J_i x J_i min-max inverses, dim i at T_off[i]
  int64_t T_off[nufft::kMaxDim];
  float* om_sorted;         // [d][M] trajectory in tile-sorted order
  double2* cheb;            // Chebyshev expansions of the coefficients in the offset (plan.cu)
  int cheb_ok[2];           // expansion used for the coefficients / their derivatives
  float2* dcoef;            // [sum_i J_i][M] d coef / d omega (allocated on first use)

  // kept for nufft_plan_set_trajectory: sort scratch, the validation flags and
  // the chunk capacity of chunks / tiles
  uint32_t* sort_keys;      // [2][M]
  int32_t* sort_vals;       // [M]
  uint32_t* sort_hist;      // [256][ceil(M / sort tile)]
  int32_t* perm2;           // [M]
  int* flags;               // [2]: om invalid, G singular
  uint32_t* cmax;           // [kMaxDim] largest |coefficient| per dimension (float bits), for the gridding scale
  int64_t chunk_cap;
  uint64_t generation;      // bumped whenever recorded graphs may be stale (drop_graphs)
  int4* red_work;           // [nbins] 2D tile-reduction work list of a single transform (plan.cu)
  int red_ctas;             // its items (0: no list; the one-tile-per-CTA reduction runs)


  // Toeplitz-embedded normal operator (nufft_toeplitz_init)
  nufft_plan* toep_geom;    // FFT geometry N in a 2N grid, no trajectory
  float2* toep_T;           // kernel spectrum / (2N)^d on the 2N grid
  float2* toep_grid;        // [batch][ (2N)^d ] work space
  int toep_cap;             // batch capacity of toep_grid
  int normal_op;            // 0: V^H V through the grid, 1: Toeplitz (solvers)

  // CUDA graphs of the entry points' launch sequences (see run_graphed)
  int graphs_enabled;
  cudaStream_t capture_stream;
  nufft::GraphEntry graphs[nufft::kGraphSlots];
  uint64_t graph_clock;

  // batched work space (grown on demand): grids, partial tiles, k-space, images
  int batch_cap;
  float2* bgrid;            // [batch_cap][Kprod]
  float2* btiles;           // [batch_cap][nchunks][padded_cells]
  float2* bytmp;            // [batch_cap][M]
  float2* bimg;             // [batch_cap][Nprod]

  char err[512];
};

namespace nufft {

// ------------------------------------------------------------------ errors
int set_error(nufft_plan_t* p, int code, const char* fmt, ...);
int cuda_check(nufft_plan_t* p, cudaError_t e, const char* what);
#define NUFFT_CUDA_TRY(p, call)                                   \
  do {                                                            \
    cudaError_t _e = (call);                                      \
    if (_e != cudaSuccess) return ::nufft::cuda_check((p), _e, #call); \
  } while (0)

// ------------------------------------------------------------------ device memory (memory.cu)
// All library-owned device buffers go through these (a test hook can make an
// allocation fail; the bytes held are counted).
cudaError_t dev_malloc_bytes(void** ptr, size_t bytes);
cudaError_t dev_free(void* ptr);
template <class T>
inline cudaError_t dev_malloc(T** ptr, size_t bytes) {
  return dev_malloc_bytes(reinterpret_cast<void**>(ptr), bytes);
}

// Group size and thread groups of the 2D tile reduction of one transform
// (tiles of `cells` cells); shared by the launcher and the plan's work list.
inline void reduce2d_groups(int cells, int* gsize, int* ng) {
  *gsize = std::max(32, std::min(1024, (cells + 127) / 128 * 32));
  *ng = std::max(1, std::min(4, 1024 / *gsize));
}

// ------------------------------------------------------------------ launchers
// Work of a CG step folded into the image-side FFT passes of a normal
// operator q = A^H A p (single transforms only; solvers.cu):
//  pro_*: the forward pass that reads the image first updates it in place,
//    p = r + beta p, beta = (sum of pro_part[0 .. pro_count)) / pro_sc[pro_old],
//    and CTA 0 stores that sum in pro_sc[pro_new] (pro_p == NULL: no update);
//  epi_*: the inverse pass that writes the image also writes, per CTA, the
//    partial sum of Re(conj(epi_a) q) over its outputs to epi_part[blockIdx.x];
//    the launcher reports the number of CTAs in *epi_count (at most epi_cap,
//    else NUFFT_EINVAL).
// Every sum runs in a fixed order.
struct CgHooks {
  float2* pro_p = nullptr;
  const float2* pro_r = nullptr;
  const double* pro_part = nullptr;
  int pro_count = 0;
  double* pro_sc = nullptr;
  int pro_old = 0, pro_new = 0;
  const float2* epi_a = nullptr;
  double* epi_part = nullptr;
  int epi_cap = 0;
  int* epi_count = nullptr;
};

// FFT passes (fft.cu).  Forward: grid = F pad(S x).  Inverse: x = S crop(F^H grid).
// nb > 1 runs nb independent transforms: images nb x N^d, grids nb x K^d.
// scale = false leaves out S (S^H): a plain centred zero-pad (crop).
int launch_fft_forward(nufft_plan_t* p, const float2* x, float2* grid, int nb = 1, bool scale = true,
                       const CgHooks* hooks = nullptr);
int launch_fft_inverse(nufft_plan_t* p, float2* grid, float2* x, int nb = 1, bool scale = true,
                       const CgHooks* hooks = nullptr);
// CTAs of the inverse pass that writes the image (single transform).
int fft_inverse_last_blocks(nufft_plan_t* p, int64_t* blocks);

// Interpolation and gridding (interp.cu).
// nb > 1: grids nb x K^d, k-space data nb x M, partial tiles in `tiles`
// (nb x nchunks x padded tile; NULL = the plan's single-batch buffer).
int launch_interp(nufft_plan_t* p, const float2* grid, float2* y, int nb = 1);
int launch_gridding(nufft_plan_t* p, const float2* y, float2* grid, int nb = 1, float2* tiles = nullptr);
// V^H V on the oversampled grid in one chunk pass (2D): grid_in -> grid_out
// (they may be the same buffer); vhv_fused tells whether the plan has it.
bool vhv_fused(const nufft_plan_t* p);
int launch_vhv(nufft_plan_t* p, const float2* grid_in, float2* grid_out, int nb = 1, float2* tiles = nullptr);

// Batched operators (capi.cu): nb transforms with one launch per stage.
int ensure_batch(nufft_plan_t* p, int nb);
int forward_batch_impl(nufft_plan_t* p, int nb, const float2* x, float2* y);
int adjoint_batch_impl(nufft_plan_t* p, int nb, const float2* y, float2* x);
int selfadjoint_batch_impl(nufft_plan_t* p, int nb, const float2* x, float2* out);

// CUDA graphs (graphs.cu).  run_graphed runs `body` (which launches work on
// p->stream) eagerly the first time a (kind, a, b, extra, stream) key is seen,
// captures it into a graph on a plan-owned stream the second time, and replays
// the graph into p->stream after that.  Work already being captured by the
// caller, or a plan with graphs disabled, runs eagerly.  Any change that frees
// plan-owned buffers must call drop_graphs.
int run_graphed_impl(nufft_plan_t* p, int kind, const void* a, const void* b, int64_t extra, int (*fn)(void*),
                     void* ctx);
template <class F>
int run_graphed(nufft_plan_t* p, int kind, const void* a, const void* b, int64_t extra, F body) {
  return run_graphed_impl(p, kind, a, b, extra, [](void* c) -> int { return (*static_cast<F*>(c))(); }, &body);
}
void drop_graphs(nufft_plan_t* p);

// `extra` of a graph key that carries several parameters: an FNV-1a hash of
// their bit patterns (pointers and doubles passed through graph_bits).
inline uint64_t graph_bits(double v) {
  uint64_t b;
  memcpy(&b, &v, 8);
  return b;
}
inline uint64_t graph_bits(const void* v) { return (uint64_t)(uintptr_t)v; }
inline int64_t graph_key(std::initializer_list<uint64_t> vals) {
  uint64_t h = 1469598103934665603ull;
  for (uint64_t v : vals) {
    h ^= v;
    h *= 1099511628211ull;
  }
  return (int64_t)h;
}

// Normal operator used by the solvers (toeplitz.cu): V^H V or Toeplitz.
int normal_op(nufft_plan_t* p, const float2* x, float2* out, int nb = 1);
// The same for one image with a CG step's work folded into its FFT passes
// (x is updated in place by the prologue), and the number of partial sums
// its epilogue writes.
int normal_op_hooked(nufft_plan_t* p, float2* x, float2* out, const CgHooks* h);
int normal_op_epi_blocks(nufft_plan_t* p, int64_t* blocks);
// A^H A x with CG hooks (capi.cu).
int selfadjoint_hooked(nufft_plan_t* p, float2* x, float2* out, const CgHooks* h);

// Plan-time helpers (plan.cu).
Points points_view(const nufft_plan_t* p);
// d coef / d omega into p->dcoef (allocated here on first use).
int ensure_coef_derivatives(nufft_plan_t* p);

}  // namespace nufft

// ------------------------------------------------------------------ complex helpers
// Grid index k0 + j wrapped into [0, K), for k0 in [0, K) and 0 <= j < K.
__host__ __device__ __forceinline__ int wrapk(int v, int K) { return v >= K ? v - K : v; }

__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // conj(a) * b
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  return make_float2(a.x + b.x, a.y + b.y);
}
// Loads of data read for the last time (a line pass's input), marked
// evict-first in L2 so that they do not push out what the launch writes for
// the next one (a 3D pass's 67 MB output stays in L2 while it streams the
// 134 MB grid in).
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ float2 ld_last_use(const float2* ptr, uint64_t pol) {
  float2 v;
  asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(ptr), "l"(pol));
  return v;
}

// acc + a * b as four fused multiply-adds (cadd(acc, cmul(a, b)) rounds the
// product before the sum and takes six instructions)
__host__ __device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
  return make_float2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) {
  return make_float2(a.x * s, a.y * s);
}
