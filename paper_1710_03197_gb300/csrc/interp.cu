// interp.cu - interpolation V (grid -> k-space) and gridding V^H
// (k-space -> grid) with the min-max interpolator.
//
// Section 2.1.3: V maps the oversampled grid to the M non-uniform points, each
// point combining its J^d neighbours; gridding is its conjugate transpose.
// The paper stores V as a CSR matrix and runs a sparse matrix-vector product
// for both directions.  Here each point keeps only its first neighbour per
// dimension and J coefficients per dimension (the d-dimensional weight is their
// product), and points are sorted by grid tile at plan time.
//
// Interpolation: a group of J_last lanes handles one point; lane l owns the
// l-th neighbour along the last (contiguous) axis, so the group reads J_last
// consecutive grid cells per neighbour row, and the partial sums are combined
// with warp shuffles.
//
// Gridding: one CTA per chunk of a tile's points accumulates conj(weight) * y
// into a shared-memory copy of the tile extended by J-1 cells per dimension
// (the "padded tile"), then writes the padded tile to a per-chunk buffer.  A
// second kernel forms every grid cell of a tile as the sum, in a fixed order,
// of the padded tiles that cover it (its own tile's chunks and those of the
// 2^d - 1 lower neighbour tiles).  No global atomics; every grid cell is
// written exactly once.
#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace nufft {
namespace {

// ---------------------------------------------------------------- interpolation
// Sum of `part` over the lanes base .. base + G - 1 of a lane group, valid in
// lane base; every lane of the warp takes part.  Groups of 6 (J = 6) sum as
// (p0 + p3) + (p1 + p4) + (p2 + p5) with three shuffle steps; other widths add
// the lanes in order.
template <int JF>
__device__ __forceinline__ float2 lane_group_sum(float2 part, int base, int G) {
  if constexpr (JF == 6) {
    float2 a, s;
    a.x = part.x + __shfl_down_sync(0xffffffffu, part.x, 3);
    a.y = part.y + __shfl_down_sync(0xffffffffu, part.y, 3);
    s.x = a.x + __shfl_down_sync(0xffffffffu, a.x, 1);
    s.y = a.y + __shfl_down_sync(0xffffffffu, a.y, 1);
    s.x += __shfl_down_sync(0xffffffffu, a.x, 2);
    s.y += __shfl_down_sync(0xffffffffu, a.y, 2);
    return s;
  } else {
    float2 tot = make_float2(0.f, 0.f);
    for (int r = 0; r < G; ++r) {
      const int src = (base + r) & 31;
      tot.x += __shfl_sync(0xffffffffu, part.x, src);
      tot.y += __shfl_sync(0xffffffffu, part.y, src);
    }
    return tot;
  }
}

template <int D, int JF>
__global__ void __launch_bounds__(256)
k_interp(const float2* __restrict__ grid_b, float2* __restrict__ y_b, const Points P, const Geom g, int64_t gbs,
         int64_t ybs) {
  const float2* __restrict__ grid = grid_b + (int64_t)blockIdx.y * gbs;
  float2* __restrict__ y = y_b + (int64_t)blockIdx.y * ybs;
  const int G = JF > 0 ? JF : g.J[D - 1];
  const int lane = threadIdx.x & 31;
  const int per_warp = 32 / G;
  const int sub = lane / G;
  const int l = lane - sub * G;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t i = warp * per_warp + sub;
  const bool active = (sub < per_warp) && (i < P.M);

  float2 part = make_float2(0.f, 0.f);
  if (active) {
    const int J0 = JF > 0 ? JF : g.J[0];
    const int J1 = JF > 0 ? JF : (D > 1 ? g.J[1] : 1);
    const int kl = P.kf[(int64_t)(D - 1) * P.M + i];
    const int Klast = g.K[D - 1];
    const int gl = wrapk(kl + l, Klast);
    const float2 cl = P.coef[P.coef_off[D - 1] + (int64_t)l * P.M + i];
    if (D == 1) {
      part = cmul(cl, __ldg(&grid[gl]));
    } else if (D == 2) {
      const int k0 = P.kf[i];
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int j0 = 0; j0 < (JF > 0 ? JF : kMaxJ); ++j0) {
        if (JF == 0 && j0 >= J0) break;
        const float2 c0 = P.coef[P.coef_off[0] + (int64_t)j0 * P.M + i];
        const int row = wrapk(k0 + j0, g.K[0]) * (int)g.Kstride[0];
        acc = cfma(c0, __ldg(&grid[row + gl]), acc);
      }
      part = cmul(cl, acc);
    } else {
      const int k0 = P.kf[i];
      const int k1 = P.kf[P.M + i];
      float2 c1v[JF > 0 ? JF : kMaxJ];
#pragma unroll
      for (int j1 = 0; j1 < (JF > 0 ? JF : kMaxJ); ++j1) {
        if (JF == 0 && j1 >= J1) break;
        c1v[j1] = P.coef[P.coef_off[1] + (int64_t)j1 * P.M + i];
      }
      // row offsets of the J1 neighbour rows within a plane (32-bit: K^d < 2^31)
      int rowoff[JF > 0 ? JF : kMaxJ];
#pragma unroll
      for (int j1 = 0; j1 < (JF > 0 ? JF : kMaxJ); ++j1) {
        if (JF == 0 && j1 >= J1) break;
        rowoff[j1] = wrapk(k1 + j1, g.K[1]) * (int)g.Kstride[1] + gl;
      }
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll 1
      for (int j0 = 0; j0 < J0; ++j0) {
        const float2 c0 = P.coef[P.coef_off[0] + (int64_t)j0 * P.M + i];
        const float2* plane = grid + wrapk(k0 + j0, g.K[0]) * (int)g.Kstride[0];
        float2 acc1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int j1 = 0; j1 < (JF > 0 ? JF : kMaxJ); ++j1) {
          if (JF == 0 && j1 >= J1) break;
          acc1 = cfma(c1v[j1], __ldg(&plane[rowoff[j1]]), acc1);
        }
        acc = cfma(c0, acc1, acc);
      }
      part = cmul(cl, acc);
    }
  }
  // Sum the G partial values of each lane group (a fixed order).
  const float2 tot = lane_group_sum<JF>(part, sub * G, G);
  if (active && l == 0) y[P.perm[i]] = tot;
}

// ---------------------------------------------------------------- interpolation, per chunk
// One CTA per chunk of a tile's points (3D; 2D below).  The chunk's padded tile of
// the grid ((T+J-1)^d cells, wrapped at the grid edge) is copied into shared
// memory once, as a plane of real parts and a plane of imaginary parts, and
// every point gathers its J^d neighbours from there instead of from global
// memory.  The plan orders each chunk so that the points sharing a warp
// instruction read disjoint bank windows of these planes (the gridding uses
// the same order for its atomics).  Lane layout, arithmetic and summation
// order are those of k_interp (results agree to rounding: the compiler may
// fuse the multiply-adds differently in the two kernels).
template <int D>
struct InterpChunkCfg {
  static constexpr int kThreads = D == 3 ? 512 : 256;
  static constexpr int kMinBlocks = D == 3 ? 2 : 4;
};

template <int D, int JF, int TF>
__global__ void __launch_bounds__(InterpChunkCfg<D>::kThreads, InterpChunkCfg<D>::kMinBlocks)
k_interp_chunk(const float2* __restrict__ grid_b, float2* __restrict__ y_b, const Chunk* __restrict__ chunks,
               const Points P, const Geom g, int64_t gbs, int64_t ybs) {
  static_assert(TF == 0 || JF > 0, "a fixed tile needs a fixed J");
  constexpr int PF = TF > 0 ? TF + JF - 1 : 0;
  extern __shared__ float tile[];
  const float2* __restrict__ grid = grid_b + (int64_t)blockIdx.y * gbs;
  float2* __restrict__ y = y_b + (int64_t)blockIdx.y * ybs;
  const int ncell = TF > 0 ? (D == 2 ? PF * PF : PF * PF * PF) : (int)g.padded_cells;
  const int P1 = TF > 0 ? PF : g.P[1];
  const int P2 = D > 2 ? (TF > 0 ? PF : g.P[2]) : 1;
  float* gre = tile;
  float* gim = tile + ncell;
  const Chunk ch = chunks[blockIdx.x];
  int org[kMaxDim];
  {
    int rem = ch.bin;
    for (int a = D - 1; a >= 0; --a) {
      org[a] = (rem % g.nb[a]) * g.T[a];
      rem /= g.nb[a];
    }
  }
  // the padded tile, cell c = (r0, r1[, r2]) in C order with pitches P
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    int r0, r1, r2 = 0;
    if (D == 2) {
      r1 = c % P1;
      r0 = c / P1;
    } else {
      r2 = c % P2;
      r1 = (c / P2) % P1;
      r0 = c / (P2 * P1);
    }
    int64_t gi = (int64_t)wrapk(org[0] + r0, g.K[0]) * g.Kstride[0] + (int64_t)wrapk(org[1] + r1, g.K[1]) * g.Kstride[1];
    if (D == 3) gi += wrapk(org[2] + r2, g.K[2]);
    const float2 v = __ldg(&grid[gi]);
    gre[c] = v.x;
    gim[c] = v.y;
  }
  __syncthreads();

  const int G = JF > 0 ? JF : g.J[D - 1];
  const int lane = threadIdx.x & 31;
  const int per_warp = 32 / G;
  const int sub = lane / G;
  const int l = lane - sub * G;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int J0 = JF > 0 ? JF : g.J[0];
  const int J1 = JF > 0 ? JF : (D > 2 ? g.J[1] : 1);
  // warp-uniform rounds of per_warp points (the lane-group sum is a full-warp shuffle)
  for (int qb = warp * per_warp; qb < ch.count; qb += nwarps * per_warp) {
    const int q = qb + sub;
    const bool act = (sub < per_warp) && (q < ch.count);
    const int64_t i = (int64_t)ch.start + q;
    float2 part = make_float2(0.f, 0.f);
    if (act) {
      const int ll = P.kf[(int64_t)(D - 1) * P.M + i] - org[D - 1] + l;
      const float2 cl = P.coef[P.coef_off[D - 1] + (int64_t)l * P.M + i];
      const int l0 = P.kf[i] - org[0];
      float2 acc = make_float2(0.f, 0.f);
      if (D == 2) {
#pragma unroll
        for (int j0 = 0; j0 < (JF > 0 ? JF : kMaxJ); ++j0) {
          if (JF == 0 && j0 >= J0) break;
          const float2 c0 = P.coef[P.coef_off[0] + (int64_t)j0 * P.M + i];
          const int cell = (l0 + j0) * P1 + ll;
          acc = cfma(c0, make_float2(gre[cell], gim[cell]), acc);
        }
      } else {
        const int l1 = P.kf[P.M + i] - org[1];
        float2 c1v[JF > 0 ? JF : kMaxJ];
#pragma unroll
        for (int j1 = 0; j1 < (JF > 0 ? JF : kMaxJ); ++j1) {
          if (JF == 0 && j1 >= J1) break;
          c1v[j1] = P.coef[P.coef_off[1] + (int64_t)j1 * P.M + i];
        }
        constexpr int kU0 = TF > 0 ? JF : 1;
#pragma unroll kU0
        for (int j0 = 0; j0 < J0; ++j0) {
          const float2 c0 = P.coef[P.coef_off[0] + (int64_t)j0 * P.M + i];
          const int rowbase = ((l0 + j0) * P1 + l1) * P2 + ll;
          float2 acc1 = make_float2(0.f, 0.f);
#pragma unroll
          for (int j1 = 0; j1 < (JF > 0 ? JF : kMaxJ); ++j1) {
            if (JF == 0 && j1 >= J1) break;
            const int cell = rowbase + j1 * P2;
            acc1 = cfma(c1v[j1], make_float2(gre[cell], gim[cell]), acc1);
          }
          acc = cfma(c0, acc1, acc);
        }
      }
      part = cmul(cl, acc);
    }
    const float2 tot = lane_group_sum<JF>(part, sub * G, G);
    if (act && l == 0) y[P.perm[i]] = tot;
  }
}

// 3D, J = 6, 16^3 tiles: as k_interp_chunk, and the point data are staged too,
// kSub points at a time (two threads per point: first neighbours, the 18
// coefficients, the permutation), so every global load of point data is a
// coalesced row of consecutive points and the gathers read only shared
// memory.  kSub = 160 points fill two rounds of the 16 warps' lane groups and
// keep two CTAs per SM (74 KB tile + 25 KB point data each).
constexpr int kSub3 = 160;
__global__ void __launch_bounds__(512, 2)
k_interp_chunk3d(const float2* __restrict__ grid_b, float2* __restrict__ y_b, const Chunk* __restrict__ chunks,
                 const Points P, const Geom g, int64_t gbs, int64_t ybs) {
  constexpr int JF = 6, PF = 21, ncell = PF * PF * PF;
  extern __shared__ float tile[];
  const float2* __restrict__ grid = grid_b + (int64_t)blockIdx.y * gbs;
  float2* __restrict__ y = y_b + (int64_t)blockIdx.y * ybs;
  float* gre = tile;
  float* gim = tile + ncell;
  float2* s_c0 = reinterpret_cast<float2*>(tile + 2 * ncell);   // [JF][kSub3] (2 * ncell floats: 8-byte aligned)
  float2* s_c1 = s_c0 + JF * kSub3;                              // [JF][kSub3]
  float2* s_c2 = s_c1 + JF * kSub3;                              // [kSub3][JF]
  int* s_k = reinterpret_cast<int*>(s_c2 + JF * kSub3);          // [3][kSub3]
  int* s_p = s_k + 3 * kSub3;                                    // [kSub3]
  const Chunk ch = chunks[blockIdx.x];
  int org[3];
  {
    int rem = ch.bin;
    for (int a = 2; a >= 0; --a) {
      org[a] = (rem % g.nb[a]) * 16;
      rem /= g.nb[a];
    }
  }
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const int r2 = c % PF, r1 = (c / PF) % PF, r0 = c / (PF * PF);
    const int64_t gi = (int64_t)wrapk(org[0] + r0, g.K[0]) * g.Kstride[0] +
                       (int64_t)wrapk(org[1] + r1, g.K[1]) * g.Kstride[1] + wrapk(org[2] + r2, g.K[2]);
    const float2 v = __ldg(&grid[gi]);
    gre[c] = v.x;
    gim[c] = v.y;
  }
  const int lane = threadIdx.x & 31;
  const int per_warp = 32 / JF;
  const int sub = lane / JF;
  const int l = lane - sub * JF;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  for (int s0 = 0; s0 < ch.count; s0 += kSub3) {
    const int cnt = min(kSub3, ch.count - s0);
    __syncthreads();   // the tile is staged; the previous sub-chunk's data are consumed
    {
      // two threads per point: half 0 loads c0 and the first neighbours, half 1 c1, c2 and the permutation
      const int q = threadIdx.x % kSub3, half = threadIdx.x / kSub3;
      if (half < 2 && q < cnt) {
        const int64_t i = (int64_t)ch.start + s0 + q;
        if (half == 0) {
#pragma unroll
          for (int r = 0; r < JF; ++r) s_c0[r * kSub3 + q] = P.coef[P.coef_off[0] + (int64_t)r * P.M + i];
#pragma unroll
          for (int a = 0; a < 3; ++a) s_k[a * kSub3 + q] = P.kf[(int64_t)a * P.M + i] - org[a];
        } else {
#pragma unroll
          for (int r = 0; r < JF; ++r) s_c1[r * kSub3 + q] = P.coef[P.coef_off[1] + (int64_t)r * P.M + i];
#pragma unroll
          for (int r = 0; r < JF; ++r) s_c2[q * JF + r] = P.coef[P.coef_off[2] + (int64_t)r * P.M + i];
          s_p[q] = P.perm[i];
        }
      }
    }
    __syncthreads();
    for (int qb = warp * per_warp; qb < cnt; qb += nwarps * per_warp) {
      const int q = qb + sub;
      const bool act = (sub < per_warp) && (q < cnt);
      float2 part = make_float2(0.f, 0.f);
      if (act) {
        const int ll = s_k[2 * kSub3 + q] + l;
        const int l0 = s_k[q], l1 = s_k[kSub3 + q];
        float2 c1v[JF];
#pragma unroll
        for (int j1 = 0; j1 < JF; ++j1) c1v[j1] = s_c1[j1 * kSub3 + q];
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int j0 = 0; j0 < JF; ++j0) {
          const int rowbase = ((l0 + j0) * PF + l1) * PF + ll;
          float2 acc1 = make_float2(0.f, 0.f);
#pragma unroll
          for (int j1 = 0; j1 < JF; ++j1) {
            const int cell = rowbase + j1 * PF;
            acc1 = cfma(c1v[j1], make_float2(gre[cell], gim[cell]), acc1);
          }
          acc = cfma(s_c0[j0 * kSub3 + q], acc1, acc);
        }
        part = cmul(s_c2[q * JF + l], acc);
      }
      const float2 tot = lane_group_sum<6>(part, sub * JF, JF);
      if (act && l == 0) y[s_p[q]] = tot;
    }
  }
}

// 2D: the chunk's point data are staged too (one thread per point: first
// neighbours, the J0 + J1 coefficients and the permutation), so the CTA waits
// for one round of global loads instead of one per pass of its warps over the
// chunk; the gathers then read only shared memory.  Shared memory: the two
// planes of the padded tile, c0[J0][cap], c1[cap][J1] (as in the gridding's
// staged kernel), k[2][cap], perm[cap].
template <int JF>
__global__ void __launch_bounds__(256, 4)
k_interp_chunk2d(const float2* __restrict__ grid_b, float2* __restrict__ y_b, const Chunk* __restrict__ chunks,
                 const Points P, const Geom g, int64_t gbs, int64_t ybs) {
  constexpr int cap = kChunkPoints[2];
  static_assert(cap == 256, "one thread per staged point");
  extern __shared__ float tile[];
  const float2* __restrict__ grid = grid_b + (int64_t)blockIdx.y * gbs;
  float2* __restrict__ y = y_b + (int64_t)blockIdx.y * ybs;
  const int ncell = (int)g.padded_cells;
  const int P1 = g.P[1];
  const int J0 = JF > 0 ? JF : g.J[0];
  const int J1 = JF > 0 ? JF : g.J[1];
  float* gre = tile;
  float* gim = tile + ncell;
  float2* s_c = reinterpret_cast<float2*>(tile + 2 * ncell);   // 8-byte aligned: 2 * ncell floats
  int* s_k = reinterpret_cast<int*>(s_c + (J0 + J1) * cap);
  int* s_p = s_k + 2 * cap;
  const Chunk ch = chunks[blockIdx.x];
  const int org0 = ((ch.bin / g.nb[1]) % g.nb[0]) * g.T[0];
  const int org1 = (ch.bin % g.nb[1]) * g.T[1];
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const int r1 = c % P1, r0 = c / P1;
    const float2 v = __ldg(&grid[(int64_t)wrapk(org0 + r0, g.K[0]) * g.Kstride[0] + wrapk(org1 + r1, g.K[1])]);
    gre[c] = v.x;
    gim[c] = v.y;
  }
  const int qs = threadIdx.x;
  if (qs < ch.count) {
    const int64_t i = (int64_t)ch.start + qs;
    s_p[qs] = P.perm[i];
    s_k[qs] = P.kf[i] - org0;
    s_k[cap + qs] = P.kf[P.M + i] - org1;
#pragma unroll
    for (int r = 0; r < (JF > 0 ? JF : kMaxJ); ++r) {
      if (JF == 0 && r >= J0) break;
      s_c[r * cap + qs] = P.coef[P.coef_off[0] + (int64_t)r * P.M + i];
    }
#pragma unroll
    for (int r = 0; r < (JF > 0 ? JF : kMaxJ); ++r) {
      if (JF == 0 && r >= J1) break;
      s_c[J0 * cap + qs * J1 + r] = P.coef[P.coef_off[1] + (int64_t)r * P.M + i];
    }
  }
  __syncthreads();

  const int G = J1;
  const int lane = threadIdx.x & 31;
  const int per_warp = 32 / G;
  const int sub = lane / G;
  const int l = lane - sub * G;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  for (int qb = warp * per_warp; qb < ch.count; qb += nwarps * per_warp) {
    const int q = qb + sub;
    const bool act = (sub < per_warp) && (q < ch.count);
    float2 part = make_float2(0.f, 0.f);
    if (act) {
      const int ll = s_k[cap + q] + l;
      const int l0 = s_k[q];
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int j0 = 0; j0 < (JF > 0 ? JF : kMaxJ); ++j0) {
        if (JF == 0 && j0 >= J0) break;
        const int cell = (l0 + j0) * P1 + ll;
        acc = cfma(s_c[j0 * cap + q], make_float2(gre[cell], gim[cell]), acc);
      }
      part = cmul(s_c[J0 * cap + q * J1 + l], acc);
    }
    const float2 tot = lane_group_sum<JF>(part, sub * G, G);
    if (act && l == 0) y[s_p[q]] = tot;
  }
}

// ---------------------------------------------------------------- gridding, per chunk
// Deterministic accumulation.  The points of a chunk add into a shared copy
// of the padded tile in fixed point: every contribution is scaled by a power
// of two S chosen per chunk (and batch element), rounded to an integer and
// added with a 32-bit integer atomic.  Integer addition is exact and
// associative, so the padded tile does not depend on the order in which the
// warps' atomics land, and two runs give bit-identical grids.  S comes from
// a bound on every cell's sum of magnitudes,
//   B = cbound * sum over the chunk's points of (|Re y| + |Im y|),
// cbound = prod_d max |c_d| (a point adds to a cell at most once), taken in a
// fixed order, so S is the same on every run too:
//   1D, 2D (chunks of <= 1024, <= 256 points): one int32 word per component,
//     sums below 2^30 (S = 2^(30 - E), B < 2^E); a contribution's rounding
//     error is at most 2^-31 B;
//   3D (chunks of <= 2048 points): 2^34 of range in three words per cell: the
//     part above 2^20 of both components packed as two 16-bit fields of one
//     word (|sum| <= 2^14 + 1024 each), and the remainders below 2^20 in one
//     word each (|sum| <= 2048 * 2^19); rounding error at most 2^-35 B.
// A chunk whose bound is not finite (an Inf or NaN sample) writes NaN.
template <int D>
struct Fix {
  static constexpr int kBits = D == 3 ? 34 : 30;   // range of a cell's sum, log2
  static constexpr int kWords = D == 3 ? 3 : 2;    // int32 words per cell
};

// Sum of v over the CTA in a fixed order (shuffle tree, then warps in order);
// every thread gets the sum.  red: 32 floats of shared scratch.
__device__ __forceinline__ float block_sum_fixed(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  for (int w = 0; w < nw; ++w) t += red[w];
  __syncthreads();   // red free for reuse
  return t;
}

struct ChunkScale {
  float S, inv;   // power-of-two scale and its inverse
  bool finite;
};

template <int D>
__device__ __forceinline__ ChunkScale chunk_scale(float ysum, const uint32_t* cmax) {
  float cb = 1.f;
#pragma unroll
  for (int a = 0; a < D; ++a) cb *= __uint_as_float(__ldg(&cmax[a]));
  const float B = ysum * cb;
  ChunkScale cs;
  cs.finite = isfinite(B);
  int E = 0;
  frexpf(cs.finite ? B : 0.f, &E);                   // B < 2^E
  E = max(E, Fix<D>::kBits - 126);                   // keep S and 1/S normal floats
  cs.S = ldexpf(1.f, Fix<D>::kBits - E);
  cs.inv = ldexpf(1.f, E - Fix<D>::kBits);
  return cs;
}

// Add one contribution w (already scaled by S) to cell `cell`.
//   D < 3: acc[0][cell] += rn(Re w), acc[1][cell] += rn(Im w)
//   D = 3: packed high parts in acc[0], remainders in acc[1], acc[2]
template <int D>
__device__ __forceinline__ void fix_add(int* acc, int ncell, int cell, float2 w) {
  if (D < 3) {
    atomicAdd(&acc[cell], __float2int_rn(w.x));
    atomicAdd(&acc[ncell + cell], __float2int_rn(w.y));
  } else {
    // x + 1.5 * 2^23 rounds x to an integer when |x| < 2^22, and the float's
    // bits minus those of 1.5 * 2^23 are that integer (the high parts); the
    // exact remainders are rounded by the conversion unit (the same
    // round-to-nearest-even), one instruction each on an otherwise idle pipe.
    const float magic = 12582912.0f;
    const float hr = fmaf(w.x, 0x1p-20f, magic), hi_ = fmaf(w.y, 0x1p-20f, magic);
    const float lr = fmaf(-(hr - magic), 0x1p20f, w.x);   // remainder (exact)
    const float li = fmaf(-(hi_ - magic), 0x1p20f, w.y);
    const int hre = __float_as_int(hr) - 0x4B400000, him = __float_as_int(hi_) - 0x4B400000;
    atomicAdd(&acc[cell], him * 65536 + hre);
    atomicAdd(&acc[ncell + cell], __float2int_rn(lr));
    atomicAdd(&acc[2 * ncell + cell], __float2int_rn(li));
  }
}

// Value of cell c of the fixed-point tile, unscaled.
template <int D>
__device__ __forceinline__ float2 fix_value(const int* acc, int ncell, int c, const ChunkScale& cs) {
  if (!cs.finite) return make_float2(__int_as_float(0x7fffffff), __int_as_float(0x7fffffff));
  if (D < 3) return make_float2((float)acc[c] * cs.inv, (float)acc[ncell + c] * cs.inv);
  const int w = acc[c];
  const int hre = (int)(short)(w & 0xffff);   // low field, sign-extended
  const int him = (w - hre) / 65536;
  const long long re = (long long)hre * 1048576 + acc[ncell + c];
  const long long im = (long long)him * 1048576 + acc[2 * ncell + c];
  return make_float2((float)re * cs.inv, (float)im * cs.inv);
}

// The accumulator words are held as planes (word k of every cell, then word
// k + 1, ...) so that the J_last lanes of a point hit J_last consecutive banks
// per atomic.
template <int D, int JF>
struct GridChunkCfg {
  static constexpr int kThreads = D == 3 ? 512 : 256;
  static constexpr int kMinBlocks = D == 3 ? 2 : 4;
};

// TF > 0: every tile edge is TF and every J is JF, so the padded-tile pitches
// are compile-time constants and the neighbour loops unroll into fixed
// shared-memory offsets.
template <int D, int JF, int TF>
__global__ void __launch_bounds__(GridChunkCfg<D, JF>::kThreads, GridChunkCfg<D, JF>::kMinBlocks)
k_gridding_chunk(const float2* __restrict__ y_b, float2* __restrict__ tiles_b, const Chunk* __restrict__ chunks,
                 const Points P, const Geom g, int64_t ybs, int64_t tbs) {
  static_assert(TF == 0 || JF > 0, "a fixed tile needs a fixed J");
  constexpr int PF = TF > 0 ? TF + JF - 1 : 0;   // padded edge when fixed
  extern __shared__ int acc[];
  __shared__ float red[32];
  const float2* __restrict__ y = y_b + (int64_t)blockIdx.y * ybs;
  float2* __restrict__ tiles = tiles_b + (int64_t)blockIdx.y * tbs;
  const int ncell = TF > 0 ? (D == 1 ? PF : (D == 2 ? PF * PF : PF * PF * PF)) : (int)g.padded_cells;
  const Chunk ch = chunks[blockIdx.x];
  for (int c = threadIdx.x; c < Fix<D>::kWords * ncell; c += blockDim.x) acc[c] = 0;

  // the chunk's scale (the sum also orders the zeroing above before the atomics)
  float part = 0.f;
  for (int q = threadIdx.x; q < ch.count; q += blockDim.x) {
    const float2 v = __ldg(&y[P.perm[(int64_t)ch.start + q]]);
    part += fabsf(v.x) + fabsf(v.y);
  }
  const ChunkScale cs = chunk_scale<D>(block_sum_fixed(part, red), P.cmax);

  // tile origin of this chunk's bin
  int org[kMaxDim];
  {
    int rem = ch.bin;
    for (int a = D - 1; a >= 0; --a) {
      org[a] = (rem % g.nb[a]) * g.T[a];
      rem /= g.nb[a];
    }
  }
  const int G = JF > 0 ? JF : g.J[D - 1];
  const int lane = threadIdx.x & 31;
  const int per_warp = 32 / G;
  const int sub = lane / G;
  const int l = lane - sub * G;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int P1 = D > 1 ? (TF > 0 ? PF : g.P[1]) : 1;
  const int P2 = D > 2 ? (TF > 0 ? PF : g.P[2]) : 1;

  // Consecutive points of the chunk share a warp instruction: the plan orders
  // each chunk so that every aligned group of per_warp points covers disjoint
  // shared-memory bank windows (see the bank-order kernel in plan.cu).
  if (sub < per_warp && cs.finite) {
    const int stepq = nwarps * per_warp;
    int q = warp * per_warp + sub;
    // 1D/2D: the dependent load (sample through the permutation) runs one
    // point ahead; 3D has enough work per point to hide it and no registers
    // to spare.
    float2 y_next = make_float2(0.f, 0.f);
    if (D < 3 && q < ch.count) y_next = __ldg(&y[P.perm[(int64_t)ch.start + q]]);
    for (; q < ch.count; q += stepq) {
      const int64_t i = (int64_t)ch.start + q;
      float2 yv;
      if (D < 3) {
        yv = y_next;
        if (q + stepq < ch.count) y_next = __ldg(&y[P.perm[i + stepq]]);
      } else {
        yv = __ldg(&y[P.perm[i]]);
      }
      yv = cscale(yv, cs.S);
      const int ll = P.kf[(int64_t)(D - 1) * P.M + i] - org[D - 1] + l;
      const float2 cl = P.coef[P.coef_off[D - 1] + (int64_t)l * P.M + i];
      const float2 yl = cmulc(cl, yv);  // conj(c_last) * y
      if (D == 1) {
        fix_add<D>(acc, ncell, ll, yl);
      } else if (D == 2) {
        const int l0 = P.kf[i] - org[0];
        const int J0 = JF > 0 ? JF : g.J[0];
#pragma unroll
        for (int j0 = 0; j0 < (JF > 0 ? JF : kMaxJ); ++j0) {
          if (JF == 0 && j0 >= J0) break;
          const float2 c0 = P.coef[P.coef_off[0] + (int64_t)j0 * P.M + i];
          fix_add<D>(acc, ncell, (l0 + j0) * P1 + ll, cmulc(c0, yl));
        }
      } else {
        const int l0 = P.kf[i] - org[0];
        const int l1 = P.kf[P.M + i] - org[1];
        const int J0 = JF > 0 ? JF : g.J[0];
        const int J1 = JF > 0 ? JF : g.J[1];
        float2 c1v[JF > 0 ? JF : kMaxJ];
#pragma unroll
        for (int j1 = 0; j1 < (JF > 0 ? JF : kMaxJ); ++j1) {
          if (JF == 0 && j1 >= J1) break;
          c1v[j1] = P.coef[P.coef_off[1] + (int64_t)j1 * P.M + i];
        }
        constexpr int kU0 = TF > 0 ? JF : 1;
#pragma unroll kU0
        for (int j0 = 0; j0 < J0; ++j0) {
          const float2 c0 = P.coef[P.coef_off[0] + (int64_t)j0 * P.M + i];
          const float2 w0 = cmulc(c0, yl);
          const int rowbase = ((l0 + j0) * P1 + l1) * P2 + ll;
#pragma unroll
          for (int j1 = 0; j1 < (JF > 0 ? JF : kMaxJ); ++j1) {
            if (JF == 0 && j1 >= J1) break;
            fix_add<D>(acc, ncell, rowbase + j1 * P2, cmulc(c1v[j1], w0));
          }
        }
      }
    }
  }
  __syncthreads();
  float2* out = tiles + (int64_t)blockIdx.x * g.padded_cells;
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) out[c] = fix_value<D>(acc, ncell, c, cs);
}

// ---------------------------------------------------------------- gridding, tile reduction
// One CTA per tile: grid cell c of tile b is the sum over e in {0,1}^d of the
// padded tiles of bin b - e (wrapped per dimension) at local position
// c - origin(b) + e * T, when that position lies inside the padded tile.  Each
// thread owns CPT cells of the tile; their padded-tile offset and the mask of
// neighbours e that reach them are computed once, so every (e, chunk) pair
// costs one predicated load per cell.  The sum runs over e, then over the
// source bin's chunks, in a fixed order.
// The whole CTA reduces grid tile `bin`; `part` is shared scratch of
// blockDim.x * CPT values.
// The cells reduced are cbase .. cbase + (blockDim/NG)*CPT - 1 of the tile (all
// of it when cbase = 0 and the groups span it).
// Entry n (2^D bits at bit 2^D * n) is the set of the e in [0, 2^D) with
// e & ~n == 0: the neighbours whose padded tiles reach a cell that is near the
// low edge of its tile along the axes in n.
template <int D>
__host__ __device__ constexpr uint64_t subset_masks() {
  uint64_t t = 0;
  for (unsigned n = 0; n < (1u << D); ++n)
    for (unsigned e = 0; e < (1u << D); ++e)
      if ((e & ~n) == 0) t |= uint64_t(1) << ((1u << D) * n + e);
  return t;
}

// Per-cell set-up of a tile reduction: the thread's CPT cells are
// cbase + tg + k * gsize of tile bc (coordinates in tiles); loc0 is a cell's
// offset in a padded tile, emask the neighbours e whose padded tiles reach it
// (0 beyond cend), goff its grid offset.
template <int D, int CPT, int TF>
__device__ __forceinline__ void reduce_cells(const Geom& g, const int (&bc)[kMaxDim], int cbase, int tg, int gsize,
                                             int tile_cells, int cend, int (&loc0)[CPT], unsigned (&emask)[CPT],
                                             int (&goff)[CPT]) {
  const int P1 = D > 1 ? g.P[1] : 1, P2 = D > 2 ? g.P[2] : 1;
  // TF > 0: every tile edge is TF, so the cell decompositions below divide by constants
  const int T1 = D > 1 ? (TF > 0 ? TF : g.T[1]) : 1, T2 = D > 2 ? (TF > 0 ? TF : g.T[2]) : 1;
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int c = min(cbase + tg + k * gsize, tile_cells - 1);
    int lc[3] = {0, 0, 0};
    if (D == 1) {
      lc[0] = c;
    } else if (D == 2) {
      lc[1] = c % T1;
      lc[0] = c / T1;
    } else {
      lc[2] = c % T2;
      lc[1] = (c / T2) % T1;
      lc[0] = c / (T2 * T1);
    }
    loc0[k] = D == 1 ? lc[0] : (D == 2 ? lc[0] * P1 + lc[1] : (lc[0] * P1 + lc[1]) * P2 + lc[2]);
    // neighbour e reaches the cell iff every axis a with e_a = 1 has the cell
    // within J - 1 of the tile's low edge; with those axes as the bits of
    // `near` (e's bit order), the mask is the set of subsets of near
    unsigned near = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) near |= (lc[a] + g.T[a] < g.P[a] ? 1u : 0u) << (D - 1 - a);
    const unsigned m = (unsigned)(subset_masks<D>() >> ((1 << D) * near)) & ((1u << (1 << D)) - 1u);
    emask[k] = (cbase + tg + k * gsize < cend) ? m : 0u;
    int off = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) off += (bc[a] * g.T[a] + lc[a]) * (int)g.Kstride[a];
    goff[k] = off;
  }
}

template <int D, int CPT, int TF>
__device__ __forceinline__ void reduce_tile(const float2* __restrict__ tiles, const int32_t* __restrict__ bin_chunk,
                                            float2* __restrict__ grid, const Geom& g, const int NG, const int bin,
                                            float2* part, const int cbase = 0) {
  // NG thread groups of blockDim/NG threads; group h takes every NG-th (e, chunk)
  // pair, and the groups' sums are added in group order at the end.
  __shared__ int s_q0[1 << kMaxDim], s_q1[1 << kMaxDim], s_delta[1 << kMaxDim];
  int bc[kMaxDim];
  {
    int rem = bin;
#pragma unroll
    for (int a = D - 1; a >= 0; --a) {
      bc[a] = rem % g.nb[a];
      rem /= g.nb[a];
    }
  }
  const int P1 = D > 1 ? g.P[1] : 1, P2 = D > 2 ? g.P[2] : 1;
  if (threadIdx.x < (1 << D)) {
    const int e = threadIdx.x;
    int src = 0, delta = 0;
    for (int a = 0; a < D; ++a) {
      const int ea = (e >> (D - 1 - a)) & 1;
      src = src * g.nb[a] + (bc[a] - ea + g.nb[a]) % g.nb[a];
      const int pstride = a == D - 1 ? 1 : (a == D - 2 ? g.P[D - 1] : P1 * P2);
      delta += ea * g.T[a] * pstride;
    }
    s_q0[e] = bin_chunk[src];
    s_q1[e] = bin_chunk[src + 1];
    s_delta[e] = delta;
  }
  __syncthreads();
  int loc0[CPT];
  unsigned emask[CPT];
  int goff[CPT];
  float2 acc[CPT];
  int tile_cells = 1;
  for (int a = 0; a < D; ++a) tile_cells *= TF > 0 ? TF : g.T[a];
  const int gsize = blockDim.x / NG;
  const int h = threadIdx.x / gsize;
  const int tg = threadIdx.x - h * gsize;
  // A tile with few (neighbour, chunk) pairs is summed by group 0 alone; the
  // other groups then skip their set-up (CTA-uniform decision).
  int npairs = 0;
  for (int e = 0; e < (1 << D); ++e) npairs += s_q1[e] - s_q0[e];
  const int NGe = npairs > 2 * (1 << D) ? NG : 1;
  const bool active = h < NGe;
  const int cend = min(tile_cells, cbase + gsize * CPT);
#pragma unroll
  for (int k = 0; k < CPT; ++k) acc[k] = make_float2(0.f, 0.f);
  reduce_cells<D, CPT, TF>(g, bc, cbase, tg, gsize, tile_cells, cend, loc0, emask, goff);
  const int64_t pc = g.padded_cells;
  if (active) {
    int idx = 0;  // running index over the (e, chunk) pairs
#pragma unroll
    for (int e = 0; e < (1 << D); ++e) {
      const int q0 = s_q0[e], q1 = s_q1[e];
      const int delta = s_delta[e];
      // first pair of this e that belongs to group h
      int q = q0 + ((h - idx) % NGe + NGe) % NGe;
      // DEPTH pairs per step: all their loads are in flight before the adds,
      // which keep the pair order (acc + v(q) + v(q + NGe) + ...)
      constexpr int DEPTH = 2;
      for (; q + (DEPTH - 1) * NGe < q1; q += DEPTH * NGe) {
        float2 v[DEPTH][CPT];
#pragma unroll
        for (int u = 0; u < DEPTH; ++u) {
          const float2* src = tiles + (int64_t)(q + u * NGe) * pc + delta;
#pragma unroll
          for (int k = 0; k < CPT; ++k) {
            const bool on = (emask[k] >> e) & 1u;
            v[u][k] = on ? __ldg(&src[loc0[k]]) : make_float2(0.f, 0.f);
          }
        }
#pragma unroll
        for (int k = 0; k < CPT; ++k)
          if ((emask[k] >> e) & 1u) {
#pragma unroll
            for (int u = 0; u < DEPTH; ++u) acc[k] = cadd(acc[k], v[u][k]);
          }
      }
      for (; q < q1; q += NGe) {
        const float2* src = tiles + (int64_t)q * pc + delta;
#pragma unroll
        for (int k = 0; k < CPT; ++k)
          if ((emask[k] >> e) & 1u) acc[k] = cadd(acc[k], __ldg(&src[loc0[k]]));
      }
      idx += q1 - q0;
    }
  }
  if (NGe > 1) {
#pragma unroll
    for (int k = 0; k < CPT; ++k) part[h * (CPT * gsize) + k * gsize + tg] = acc[k];
    __syncthreads();
    if (h == 0) {
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        float2 t = part[k * gsize + tg];
        for (int hh = 1; hh < NGe; ++hh) t = cadd(t, part[hh * (CPT * gsize) + k * gsize + tg]);
        acc[k] = t;
      }
    }
  }
  if (h == 0) {
#pragma unroll
    for (int k = 0; k < CPT; ++k)
      if (cbase + tg + k * gsize < cend) grid[goff[k]] = acc[k];
  }
  __syncthreads();   // shared scratch free for the caller
}

// CTA x reduces slice x % slices of tile x / slices (slices of blockDim/NG*CPT cells).
template <int D, int CPT, int TF>
__global__ void __launch_bounds__(1024)
k_gridding_reduce(const float2* __restrict__ tiles_b, const int32_t* __restrict__ bin_chunk,
                  float2* __restrict__ grid_b, const Geom g, const int NG, int64_t tbs, int64_t gbs, int slices) {
  extern __shared__ float2 part[];
  const int bin = blockIdx.x / slices;
  const int cbase = (blockIdx.x - bin * slices) * (blockDim.x / NG) * CPT;
  reduce_tile<D, CPT, TF>(tiles_b + (int64_t)blockIdx.y * tbs, bin_chunk, grid_b + (int64_t)blockIdx.y * gbs, g,
                             NG, bin, part, cbase);
}


// One thread group (tg = 0 .. gsize - 1, no barriers) reduces 2D grid tile
// `bin` on its own, in the order of reduce_tile with a single group: neighbour
// e outer, the source bin's chunks in order, so the tile's cells are the same
// bit for bit.  Each thread fetches the four source bins' chunk ranges itself.
template <int CPT, int TF>
__device__ __forceinline__ void reduce_tile_group2d(const float2* __restrict__ tiles,
                                                    const int32_t* __restrict__ bin_chunk, float2* __restrict__ grid,
                                                    const Geom& g, const int bin, const int tg, const int gsize) {
  int bc[kMaxDim] = {bin / g.nb[1], bin % g.nb[1], 0};
  int q0[4], q1[4], delta[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int e0 = e >> 1, e1 = e & 1;
    const int src = ((bc[0] - e0 + g.nb[0]) % g.nb[0]) * g.nb[1] + (bc[1] - e1 + g.nb[1]) % g.nb[1];
    q0[e] = __ldg(&bin_chunk[src]);
    q1[e] = __ldg(&bin_chunk[src + 1]);
    delta[e] = e0 * g.T[0] * g.P[1] + e1 * g.T[1];
  }
  const int tile_cells = TF > 0 ? TF * TF : g.T[0] * g.T[1];
  const int cend = min(tile_cells, gsize * CPT);
  int loc0[CPT];
  unsigned emask[CPT];
  int goff[CPT];
  float2 acc[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) acc[k] = make_float2(0.f, 0.f);
  reduce_cells<2, CPT, TF>(g, bc, 0, tg, gsize, tile_cells, cend, loc0, emask, goff);
  const int64_t pc = g.padded_cells;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    for (int q = q0[e]; q < q1[e]; ++q) {
      const float2* src = tiles + (int64_t)q * pc + delta[e];
#pragma unroll
      for (int k = 0; k < CPT; ++k)
        if ((emask[k] >> e) & 1u) acc[k] = cadd(acc[k], __ldg(&src[loc0[k]]));
    }
  }
#pragma unroll
  for (int k = 0; k < CPT; ++k)
    if (tg + k * gsize < cend) grid[goff[k]] = acc[k];
}

// 2D tile reduction of a single transform over a plan-time work list: item
// {t, -2, -1, -1} is a dense tile (more than 8 (neighbour, chunk) pairs),
// reduced by the whole CTA as in k_gridding_reduce; any other item holds up
// to NG sparse tiles (-1 = none), one per thread group.  Sparse tiles then
// take a quarter of the CTAs they took one per CTA, with every group busy.
template <int CPT, int TF>
__global__ void __launch_bounds__(256, 3)
k_gridding_reduce_packed2d(const float2* __restrict__ tiles, const int32_t* __restrict__ bin_chunk,
                           float2* __restrict__ grid, const int4* __restrict__ work, const Geom g, const int NG) {
  extern __shared__ float2 part[];
  const int4 w = work[blockIdx.x];
  if (w.y == -2) {   // CTA-uniform
    reduce_tile<2, CPT, TF>(tiles, bin_chunk, grid, g, NG, w.x, part, 0);
    return;
  }
  const int gsize = blockDim.x / NG;
  const int h = threadIdx.x / gsize;
  const int t = h == 0 ? w.x : (h == 1 ? w.y : (h == 2 ? w.z : w.w));
  if (t < 0) return;
  reduce_tile_group2d<CPT, TF>(tiles, bin_chunk, grid, g, t, threadIdx.x - h * gsize, gsize);
}


// 2D variant: the chunk's point data (first neighbours, coefficients, samples)
// are first copied into shared memory by all threads at once, so the CTA waits
// for two dependent global round trips (the permutation, then the samples)
// instead of one per pass of its warps over the chunk.  The accumulation then
// follows the same lane layout, bank order and fixed-point words as
// k_gridding_chunk.
// Shared memory: the two accumulator planes, then c0[J0][cap] (row by row:
// the lanes of a point read one value), c1[cap][J1] (point by point: the J1
// lanes of a point read consecutive words, so a warp's 64-bit reads of five
// points hit distinct bank pairs), y[cap], k[2][cap] (first neighbours
// relative to the tile origin), cap = chunk size.
// FUSED (V^H V, the normal operator's grid part): y_b is the oversampled
// spectrum instead of the samples; the chunk's padded tile of it is staged in
// shared memory (two float planes after the point data), and each point's y is
// first gathered from there into shared memory (the interpolation's
// arithmetic and summation order, in the scatter's lane layout), so the
// samples never leave the CTA and the coefficients are read once for both
// directions.
template <int JF, bool FUSED>
__global__ void __launch_bounds__(256, 4)
k_gridding_chunk_staged(const float2* __restrict__ y_b, float2* __restrict__ tiles_b,
                        const Chunk* __restrict__ chunks, const Points P, const Geom g, int64_t ybs, int64_t tbs) {
  constexpr int cap = kChunkPoints[2];
  extern __shared__ int acc[];
  __shared__ float red[32];
  const float2* __restrict__ y = y_b + (int64_t)blockIdx.y * ybs;
  float2* __restrict__ tiles = tiles_b + (int64_t)blockIdx.y * tbs;
  const int ncell = (int)g.padded_cells;
  const int J0 = JF > 0 ? JF : g.J[0];
  const int J1 = JF > 0 ? JF : g.J[1];
  float2* s_c = reinterpret_cast<float2*>(acc + 2 * ncell);   // 8-byte aligned: 2 * ncell words
  float2* s_y = s_c + (J0 + J1) * cap;
  int* s_k = reinterpret_cast<int*>(s_y + cap);
  float* gre = reinterpret_cast<float*>(s_k + 2 * cap);   // FUSED: the chunk's padded tile of the spectrum
  float* gim = gre + ncell;
  const Chunk ch = chunks[blockIdx.x];
  const int org0 = ((ch.bin / g.nb[1]) % g.nb[0]) * g.T[0];
  const int org1 = (ch.bin % g.nb[1]) * g.T[1];

  for (int c = threadIdx.x; c < 2 * ncell; c += blockDim.x) acc[c] = 0;
  if (FUSED) {
    const int P1 = g.P[1];
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
      const int r1 = c % P1, r0 = c / P1;
      const float2 v = __ldg(&y[(int64_t)wrapk(org0 + r0, g.K[0]) * g.Kstride[0] + wrapk(org1 + r1, g.K[1])]);
      gre[c] = v.x;
      gim[c] = v.y;
    }
  }
  static_assert(cap == 256, "one thread per staged point");
  const int qs = threadIdx.x;           // the point this thread stages
  int pm = 0;
  if (qs < ch.count) {
    const int q = qs;
    const int64_t i = (int64_t)ch.start + q;
    if (!FUSED) pm = P.perm[i];
    s_k[q] = P.kf[i] - org0;
    s_k[cap + q] = P.kf[P.M + i] - org1;
#pragma unroll
    for (int r = 0; r < (JF > 0 ? JF : kMaxJ); ++r) {
      if (JF == 0 && r >= J0) break;
      s_c[r * cap + q] = P.coef[P.coef_off[0] + (int64_t)r * P.M + i];
    }
#pragma unroll
    for (int r = 0; r < (JF > 0 ? JF : kMaxJ); ++r) {
      if (JF == 0 && r >= J1) break;
      s_c[J0 * cap + q * J1 + r] = P.coef[P.coef_off[1] + (int64_t)r * P.M + i];
    }
  }
  if (!FUSED && qs < ch.count) s_y[qs] = __ldg(&y[pm]);
  __syncthreads();

  const int G = J1;
  const int lane = threadIdx.x & 31;
  const int per_warp = 32 / G;
  const int sub = lane / G;
  const int l = lane - sub * G;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int P1 = g.P[1];
  if (FUSED) {
    // warp-uniform rounds of per_warp points: the lane-group sum is a
    // full-warp shuffle; the spectrum is read from the staged tile
    for (int qb = warp * per_warp; qb < ch.count; qb += nwarps * per_warp) {
      const int q = qb + sub;
      const bool act = (sub < per_warp) && (q < ch.count);
      float2 part = make_float2(0.f, 0.f);
      if (act) {
        const int ll = s_k[cap + q] + l;
        const int l0 = s_k[q];
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int j0 = 0; j0 < (JF > 0 ? JF : kMaxJ); ++j0) {
          if (JF == 0 && j0 >= J0) break;
          const int cell = (l0 + j0) * P1 + ll;
          a = cfma(s_c[j0 * cap + q], make_float2(gre[cell], gim[cell]), a);
        }
        part = cmul(s_c[J0 * cap + q * J1 + l], a);
      }
      const float2 yv = lane_group_sum<JF>(part, sub * G, G);
      if (act && l == 0) s_y[q] = yv;
    }
    __syncthreads();
  }
  // the chunk's scale (also orders the zeroing and staging before the atomics)
  float mag = 0.f;
  if (qs < ch.count) mag = fabsf(s_y[qs].x) + fabsf(s_y[qs].y);
  const ChunkScale cs = chunk_scale<2>(block_sum_fixed(mag, red), P.cmax);
  if (sub < per_warp && cs.finite) {
    for (int q = warp * per_warp + sub; q < ch.count; q += nwarps * per_warp) {
      const float2 yl = cmulc(s_c[J0 * cap + q * J1 + l], cscale(s_y[q], cs.S));   // conj(c_last) * y * S
      const int ll = s_k[cap + q] + l;
      const int l0 = s_k[q];
#pragma unroll
      for (int j0 = 0; j0 < (JF > 0 ? JF : kMaxJ); ++j0) {
        if (JF == 0 && j0 >= J0) break;
        fix_add<2>(acc, ncell, (l0 + j0) * P1 + ll, cmulc(s_c[j0 * cap + q], yl));
      }
    }
  }
  __syncthreads();
  float2* out = tiles + (int64_t)blockIdx.x * g.padded_cells;
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) out[c] = fix_value<2>(acc, ncell, c, cs);
}

// The reduction gives every thread 4 cells of the tile; small tiles get up to 4
// thread groups, each summing every 4th (neighbour, chunk) pair.
template <int D>
cudaError_t launch_reduce(const nufft_plan_t* p, const float2* tiles, float2* grid, int nb = 1) {
  int cells = 1;
  for (int a = 0; a < D; ++a) cells *= p->g.T[a];
  // 3D 16^3 tiles: an eighth of a tile (512 cells) per CTA of 128 threads, so
  // that many tiles' set-up, loads and stores overlap on an SM (one 1024-thread
  // CTA of 64 registers filled an SM: 1 -> 2 -> 4 -> 8 slices measured 0.909,
  // 0.887, 0.875, 0.864 ms for the kooshball's gridding; 16 no better)
  const int slices = (D == 3 && cells >= 4096) ? 8 : 1;
  const int gsize = std::max(32, std::min(1024, (cells / slices + 4 * 32 - 1) / (4 * 32) * 32));
  if ((int64_t)gsize * 4 * slices < cells) return cudaErrorInvalidValue;
  // groups splitting the chunk list; a batch (mostly sparse tiles, many CTAs)
  // runs one group per CTA so that more tiles are in flight per SM
  const int NG = (nb > 1 || slices > 1) ? 1 : std::max(1, std::min(4, 1024 / gsize));
  const size_t smem = NG > 1 ? (size_t)NG * 4 * gsize * sizeof(float2) : 0;
  bool t16 = D > 1;
  for (int a = 0; a < D; ++a) t16 = t16 && p->g.T[a] == 16;
  if constexpr (D == 2) {
    // a single transform with the plan's work list: sparse tiles packed NG to a CTA
    int gs = 0, ng = 0;
    reduce2d_groups(cells, &gs, &ng);
    if (nb == 1 && p->red_ctas > 0 && gs == gsize && ng == NG) {
      auto kern = t16 ? k_gridding_reduce_packed2d<4, 16> : k_gridding_reduce_packed2d<4, 0>;
      kern<<<(unsigned)p->red_ctas, gsize * NG, smem, p->stream>>>(tiles, p->bin_chunk, grid, p->red_work, p->g, NG);
      return cudaGetLastError();
    }
  }
  auto kern = t16 ? k_gridding_reduce<D, 4, (D > 1 ? 16 : 0)> : k_gridding_reduce<D, 4, 0>;
  kern<<<dim3((unsigned)(p->g.nbins * slices), (unsigned)nb), gsize * NG, smem, p->stream>>>(
      tiles, p->bin_chunk, grid, p->g, NG, p->nchunks * p->g.padded_cells, p->Kprod, slices);
  return cudaGetLastError();
}

bool all_j_equal(const Geom& g, int J) {
  for (int a = 0; a < g.d; ++a)
    if (g.J[a] != J) return false;
  return true;
}

template <int D>
cudaError_t interp_chunks(const nufft_plan_t* p, const float2* grid, float2* y, int nb) {
  if (p->nchunks == 0) return cudaSuccess;
  const Points P = points_view(p);
  const dim3 gd((unsigned)p->nchunks, (unsigned)nb);
  const bool j6 = all_j_equal(p->g, 6);
  bool t16 = true;
  for (int a = 0; a < D; ++a) t16 = t16 && p->g.T[a] == 16;
  if constexpr (D == 2) {
    const int sj = p->g.J[0] + p->g.J[1];
    const size_t smem = (size_t)p->g.padded_cells * 2 * sizeof(float) +
                        (size_t)kChunkPoints[2] * ((size_t)sj * sizeof(float2) + 3 * sizeof(int));
    auto kern = j6 ? k_interp_chunk2d<6> : k_interp_chunk2d<0>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<gd, kChunkPoints[2], smem, p->stream>>>(grid, y, p->chunks, P, p->g, p->Kprod, p->M);
    return cudaGetLastError();
  } else {
    if (j6 && t16) {
      const size_t smem = (size_t)21 * 21 * 21 * 2 * sizeof(float) +
                          (size_t)kSub3 * (3 * 6 * sizeof(float2) + 4 * sizeof(int));
      cudaError_t e = cudaFuncSetAttribute(k_interp_chunk3d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k_interp_chunk3d<<<gd, 512, smem, p->stream>>>(grid, y, p->chunks, P, p->g, p->Kprod, p->M);
      return cudaGetLastError();
    }
    const size_t smem = (size_t)p->g.padded_cells * 2 * sizeof(float);
    auto kern = j6 ? (t16 ? k_interp_chunk<D, 6, 16> : k_interp_chunk<D, 6, 0>) : k_interp_chunk<D, 0, 0>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<gd, InterpChunkCfg<D>::kThreads, smem, p->stream>>>(grid, y, p->chunks, P, p->g, p->Kprod, p->M);
    return cudaGetLastError();
  }
}

template <int D>
cudaError_t interp_d(const nufft_plan_t* p, const float2* grid, float2* y, int nb) {
  // single transforms gather from staged tiles; a batch keeps the per-point
  // kernel (the chunk kernel would stage each chunk's point data once per
  // batch element: the 32-coil frames' normal operator measured 2.36 -> 2.87 ms)
  if constexpr (D > 1) {
    if (nb == 1) return interp_chunks<D>(p, grid, y, nb);
  }
  const Points P = points_view(p);
  const int G = p->g.J[D - 1];
  const int per_warp = 32 / G;
  const int64_t warps = (P.M + per_warp - 1) / per_warp;
  const int64_t blocks = (warps * 32 + 255) / 256;
  if (blocks == 0) return cudaSuccess;
  const dim3 gd((unsigned)blocks, (unsigned)nb);
  auto kern = all_j_equal(p->g, 6) ? k_interp<D, 6> : k_interp<D, 0>;
  kern<<<gd, 256, 0, p->stream>>>(grid, y, P, p->g, p->Kprod, p->M);
  return cudaGetLastError();
}

// Chunk pass of V^H: one CTA per (chunk, batch element), partial tiles out.
// FUSED (2D only): y is the oversampled spectrum and the pass computes V^H V.
template <int D, bool FUSED = false>
cudaError_t launch_chunks(const nufft_plan_t* p, const float2* y, float2* tiles, int nb, int64_t ybs, int64_t tbs) {
  if (p->nchunks == 0) return cudaSuccess;
  const Points P = points_view(p);
  const dim3 gd((unsigned)p->nchunks, (unsigned)nb);
  const bool j6 = all_j_equal(p->g, 6);
  cudaError_t e;
  if constexpr (D == 2) {
    const int sj = p->g.J[0] + p->g.J[1];
    const size_t smem = (size_t)p->g.padded_cells * Fix<2>::kWords * sizeof(int) +
                        (size_t)kChunkPoints[2] * ((size_t)sj * sizeof(float2) + sizeof(float2) + 2 * sizeof(int)) +
                        (FUSED ? (size_t)p->g.padded_cells * 2 * sizeof(float) : 0);
    auto kern = j6 ? k_gridding_chunk_staged<6, FUSED> : k_gridding_chunk_staged<0, FUSED>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<gd, kChunkPoints[2], smem, p->stream>>>(y, tiles, p->chunks, P, p->g, ybs, tbs);
  } else {
    static_assert(!FUSED, "the fused V^H V pass is 2D only");
    const size_t smem = (size_t)p->g.padded_cells * Fix<D>::kWords * sizeof(int);
    constexpr int NT = GridChunkCfg<D, 6>::kThreads;
    bool t16 = D == 3;
    for (int a = 0; a < D; ++a) t16 = t16 && p->g.T[a] == 16;
    auto kern = j6 ? (t16 ? k_gridding_chunk<D, 6, (D == 3 ? 16 : 0)> : k_gridding_chunk<D, 6, 0>)
                   : k_gridding_chunk<D, 0, 0>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<gd, NT, smem, p->stream>>>(y, tiles, p->chunks, P, p->g, ybs, tbs);
  }
  return cudaGetLastError();
}

template <int D>
cudaError_t gridding_d(const nufft_plan_t* p, const float2* y, float2* grid, int nb, float2* tiles) {
  const int64_t tbs = p->nchunks * p->g.padded_cells;
  cudaError_t e = launch_chunks<D>(p, y, tiles, nb, p->M, tbs);
  if (e != cudaSuccess) return e;
  return launch_reduce<D>(p, tiles, grid, nb);
}

// ---------------------------------------------------------------- gridding without allocation
// Partial-tile scratch for nufft_gridding_static: a fixed array in device
// memory, so that call needs neither cudaMalloc nor plan-owned scratch.
constexpr int64_t kStaticTileBytes = 16ll << 20;   // 16 MiB on every GPU that loads the library
static __device__ __align__(256) float2 g_static_tiles[kStaticTileBytes / sizeof(float2)];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
float2* g_static_ptr[kMaxDevices];   // device address of g_static_tiles, per device

// Device address of the static array on the plan's device, which the caller
// has made current.  Looked up once per device (cudaGetSymbolAddress) and
// cached; the host-side name g_static_tiles is not a device address.
int static_tiles_address(nufft_plan_t* p, float2** out) {
  const int dev = p->device;
  if (dev < 0 || dev >= kMaxDevices) return set_error(p, NUFFT_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* ptr = nullptr;
    NUFFT_CUDA_TRY(p, cudaGetSymbolAddress(&ptr, g_static_tiles));
    g_static_ptr[dev] = static_cast<float2*>(ptr);
  }
  *out = g_static_ptr[dev];
  return NUFFT_OK;
}

// Makes the plan's device current for the call and puts the caller's back.
struct DeviceScope {
  int prev = -1;
  bool switched = false;
  ~DeviceScope() {
    if (switched) cudaSetDevice(prev);
  }
  cudaError_t enter(int dev) {
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess || prev == dev) return e;
    e = cudaSetDevice(dev);
    switched = e == cudaSuccess;
    return e;
  }
};

template <int D>
cudaError_t gridding_static_d(const nufft_plan_t* p, const float2* y, float2* grid, float2* tiles) {
  cudaError_t e = launch_chunks<D>(p, y, tiles, 1, 0, 0);
  if (e != cudaSuccess) return e;
  return launch_reduce<D>(p, tiles, grid);
}

}  // namespace

int launch_interp(nufft_plan_t* p, const float2* grid, float2* y, int nb) {
  cudaError_t e;
  switch (p->g.d) {
    case 1: e = interp_d<1>(p, grid, y, nb); break;
    case 2: e = interp_d<2>(p, grid, y, nb); break;
    default: e = interp_d<3>(p, grid, y, nb); break;
  }
  return e == cudaSuccess ? NUFFT_OK : cuda_check(p, e, "interpolation kernel");
}

bool vhv_fused(const nufft_plan_t* p) { return p->g.d == 2 && p->M > 0; }

int launch_vhv(nufft_plan_t* p, const float2* grid_in, float2* grid_out, int nb, float2* tiles) {
  if (!vhv_fused(p)) return set_error(p, NUFFT_EINVAL, "fused V^H V is 2D only");
  if (!tiles) tiles = p->tiles;
  const int64_t tbs = p->nchunks * p->g.padded_cells;
  cudaError_t e = launch_chunks<2, true>(p, grid_in, tiles, nb, p->Kprod, tbs);
  if (e == cudaSuccess) e = launch_reduce<2>(p, tiles, grid_out, nb);
  return e == cudaSuccess ? NUFFT_OK : cuda_check(p, e, "fused V^H V kernels");
}

int launch_gridding(nufft_plan_t* p, const float2* y, float2* grid, int nb, float2* tiles) {
  if (!tiles) tiles = p->tiles;
  cudaError_t e;
  switch (p->g.d) {
    case 1: e = gridding_d<1>(p, y, grid, nb, tiles); break;
    case 2: e = gridding_d<2>(p, y, grid, nb, tiles); break;
    default: e = gridding_d<3>(p, y, grid, nb, tiles); break;
  }
  return e == cudaSuccess ? NUFFT_OK : cuda_check(p, e, "gridding kernels");
}

}  // namespace nufft

// Gridding V^H like nufft_gridding, with the per-chunk partial tiles in the
// static device array above instead of the plan's buffer (see the header).
extern "C" int nufft_gridding_static(nufft_plan_t* p, const float* y_dev, float* grid_dev) {
  using namespace nufft;
  if (!p) return set_error(nullptr, NUFFT_EINVAL, "plan is NULL");
  if (p->M > 0 && !y_dev) return set_error(p, NUFFT_EINVAL, "y_dev is NULL");
  if (!grid_dev) return set_error(p, NUFFT_EINVAL, "grid_dev is NULL");
  const int64_t need = p->nchunks * p->g.padded_cells * (int64_t)sizeof(float2);
  if (need > kStaticTileBytes)
    return set_error(p, NUFFT_EINVAL,
                     "gridding needs %lld bytes of partial tiles, more than the %lld-byte static scratch; "
                     "use nufft_gridding", (long long)need, (long long)kStaticTileBytes);
  DeviceScope scope;   // the kernels run on the plan's stream, so on the plan's device
  NUFFT_CUDA_TRY(p, scope.enter(p->device));
  float2* tiles = nullptr;
  const int rc = static_tiles_address(p, &tiles);
  if (rc != NUFFT_OK) return rc;
  const float2* y = reinterpret_cast<const float2*>(y_dev);
  float2* grid = reinterpret_cast<float2*>(grid_dev);
  cudaError_t e;
  switch (p->g.d) {
    case 1: e = gridding_static_d<1>(p, y, grid, tiles); break;
    case 2: e = gridding_static_d<2>(p, y, grid, tiles); break;
    default: e = gridding_static_d<3>(p, y, grid, tiles); break;
  }
  return e == cudaSuccess ? NUFFT_OK : cuda_check(p, e, "static-scratch gridding kernels");
}
