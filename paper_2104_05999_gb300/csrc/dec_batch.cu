// dec_batch.cu - many instances on one mesh in one persistent launch: the
// Dirichlet value sets of one operator, the crack states of a growing disc
// population (each state zeroes the *1 of the edges it cuts, Sec. 2.5), or
// several conductivity fields (conductivity lives on the dual 2-cells,
// Sec. 2.1), solved together by mixed-precision PCG over a sparse matrix -
// multiple vector product.
//
// Vectors are stored node-major with the instances contiguous (X[i * BS + b],
// BS = padded instance count), so a gathered neighbour row X[c][0..BS) is one
// contiguous load.  Each thread handles four consecutive instances of a row
// (16-byte loads): TPR = BS / 4 threads share a row and a warp covers
// C = 32 / TPR rows.
//
// The batched solve numbers the nodes in the Morton order of their
// coordinates (vectors, rows and columns alike; results are mapped back).
// Matrices are stored sliced (slices of C rows, entry j of the slice's rows
// contiguous), so a warp's structure loads are coalesced, and the slices are
// grouped in windows of R = 1024 / TPR consecutive rows of that order: a
// block works on one window at a time, a compact patch of the mesh whose
// neighbour rows stay in the SM's L1 while the block gathers them, and whose
// own rows are contiguous in memory.  Rows inside a window are sorted by
// length, so a slice is padded to nearly its rows' own lengths.
//
// Operator of instance b, by kind:
//   Dirichlet sets  one L for all: CSR form, y_i = L_ii x_i + sum_c L_ic x_c
//                   over free columns c (Dirichlet columns moved to b);
//   crack states    edge form from the uncracked *1 and each entry's first
//                   crack state: y_i = sum_k m_k (x_i - x_c),
//                   m_k = w_k [b < fc_k];
//   fields          edge form with a *1 per instance and entry.
// Vectors are zero on Dirichlet nodes (identity rows with b = 0), so those
// columns drop out of the edge form; a row whose weights are all zero in an
// instance (and every Dirichlet row, which stores no entries) is an identity
// row.  Dirichlet sets share one FSAI factor; crack states and fields get
// one factor each, computed in FP32 and stored in BF16 with the instances
// contiguous.
//
// Per-instance convergence masks: an instance stops working once its FP64
// residual reaches rtol; within a segment it is frozen once its FP32
// residual has dropped by the segment factor, and when no instance is left
// iterating all of them get a reliable update (x64 += x, FP64 residual
// replaced) together.  Every reduction is per instance and in a fixed order,
// so all blocks hold identical scalars and take identical branches.  Grid
// barriers spin a bounded number of times (DEC_ERR_TIMEOUT after that).
#include "dec_kern.cuh"

#include <algorithm>
#include <cmath>

namespace dec {

constexpr int kBBlock = 1024;             // one block of 1024 threads per SM
constexpr int kBWarps = kBBlock / 32;     // = slices per window
constexpr int kBMax = 64;                 // instances per batched launch
constexpr long kBSpinLimit = 1L << 24;
constexpr int kIPT = 4;                   // instances per thread

enum { kSets = 0, kStates = 1, kFields = 2 };

struct BatchArgs {
  int64_t n;
  int B, BS, TPR, C;
  int64_t nwin;                           // windows of 32 slices
  // L: slices (perm, sptr) and entries
  const int32_t* Lperm;
  const int32_t* Lsptr;
  const int2* Lcw;                        // (column, FP32 value bits): sets, states
  const uint8_t* Lfc;                     // first crack state (states)
  const int32_t* Lcol;                    // columns (fields)
  const float* Lw;                        // [total][BS] (fields)
  const double* L64;                      // FP64 values, [total] or [total][BS]
  const float* d32;                       // diagonal (sets)
  const double* d64;
  // FSAI halves: lower (G) and upper (G^T)
  const int32_t* Gperm[2];
  const int32_t* Gsptr[2];
  const int32_t* Gcol[2];
  const __nv_bfloat16* Gv[2];             // shared factor
  const __nv_bfloat16* Gb[2];             // [total][BS] per instance, or nullptr
  const double* bvec;                     // [n][BS]
  double *x64, *r64;                      // [n][BS]
  float *x, *r, *z, *p, *q, *t;           // [n][BS]
  double* partial;                        // [2][grid][BS]
  unsigned* bar;
  int* status;                            // [0] error
  int* iters;                             // [BS]
  double* result;                         // [BS] final rr, [BS] |b|^2
  double rtol2, seg2;
  int max_iter;
  int warm;                               // start from x64 (the last solution)
};

__device__ __forceinline__ bool bgrid_sync(unsigned* bar, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      // bar[2] != 0 replaces the poll limit (the context's barrier test)
      const unsigned lim = *(volatile unsigned*)(bar + 2);
      const long limit = lim ? (long)lim : kBSpinLimit;
      long polls = 0;
      unsigned ns = 32;
      while (*gen == g) {
        if (++polls > limit || *(volatile int*)err) {
          atomicExch(err, 1);
          break;
        }
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)err == 0;
}

// Per-instance state, identical in every block (kept in shared memory).
struct BState {
  double rz[kBMax], tol2[kBMax], best[kBMax], bnorm2[kBMax];
  double red[kBMax];             // result of the last reduction
  float alpha[kBMax], beta[kBMax];
  int active[kBMax];             // still solving
  int iterating[kBMax];          // active and not frozen in this segment
  int restart[kBMax];
  int stall[kBMax];
  int iters[kBMax];
  int count;                     // scratch: number of iterating instances
};

// Per-instance grid reduction; thread (r, q) of a warp contributes v[j] to
// instance 4q + j.  Lanes of equal q are summed by shuffles, the 32 warps'
// sums by one warp per instance, the blocks' partials by one warp per
// instance after the grid barrier (lane l adds partials l, l + 32, ...), all
// in a fixed order.  The result lands in S.red[b], identical in every block.
__device__ bool breduce(const double (&v)[kIPT], const BatchArgs& a, int& parity, BState& S,
                        double (*shw)[kBMax], int* err) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int TPR = a.TPR, BS = a.BS, G = gridDim.x;
#pragma unroll
  for (int j = 0; j < kIPT; ++j) {
    double x = v[j];
    for (int o = 16; o >= TPR; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane < TPR) shw[warp][kIPT * lane + j] = x;
  }
  __syncthreads();
  double* part = a.partial + (size_t)parity * G * BS;
  parity ^= 1;
  for (int b = warp; b < BS; b += kBWarps) {
    const double x = warp_sum(shw[lane][b]);
    if (lane == 0) part[(size_t)blockIdx.x * BS + b] = x;
  }
  if (!bgrid_sync(a.bar, err)) return false;
  for (int b = warp; b < BS; b += kBWarps) {
    double x = 0.0;
    for (int blk = lane; blk < G; blk += 32) x += __ldcg(part + (size_t)blk * BS + b);
    x = warp_sum(x);
    if (lane == 0) S.red[b] = x;
  }
  __syncthreads();
  return true;
}

__device__ __forceinline__ float get4(const float4& v, int j) {
  return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}
__device__ __forceinline__ void set4(float4& v, int j, float x) {
  if (j == 0) v.x = x; else if (j == 1) v.y = x; else if (j == 2) v.z = x; else v.w = x;
}

// ---------------------------------------------------------- row products
// Lane (r, q) of a warp works on row slot r of the warp's slice and on the
// instances 4q..4q+3.  Entries are taken U at a time: U coalesced structure
// loads, then U independent 16-byte gathers, then the FMAs.  The slice
// width is uniform across the warp, so the guards never diverge; padding
// entries carry value 0 and the row's own column.

// (L_b x)_i, FP32, for the four instances of lane (r, q)
template <int KIND, int U>
__device__ __forceinline__ float4 l_row(const BatchArgs& a, int64_t s, int r, int q,
                                        int32_t row, const int (&st)[kIPT],
                                        const float4* __restrict__ X) {
  const int C = a.C, TPR = a.TPR;
  const int32_t base = a.Lsptr[s];
  const int32_t W = (a.Lsptr[s + 1] - base) / C;
  const int32_t rr = row >= 0 ? row : 0;
  const float4 xi = X[(int64_t)rr * TPR + q];
  if constexpr (KIND == kSets) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int32_t j = 0; j < W; j += U) {
      int2 e[U];
      float4 xv[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        e[u] = j + u < W ? __ldg(a.Lcw + base + C * (j + u) + r) : make_int2(rr, 0);
#pragma unroll
      for (int u = 0; u < U; ++u)
        xv[u] = j + u < W ? X[(int64_t)e[u].x * TPR + q] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (j + u < W) {
          const float v = __int_as_float(e[u].y);
          acc.x = fmaf(v, xv[u].x, acc.x);
          acc.y = fmaf(v, xv[u].y, acc.y);
          acc.z = fmaf(v, xv[u].z, acc.z);
          acc.w = fmaf(v, xv[u].w, acc.w);
        }
      }
    }
    const float d = a.d32[rr];
    return make_float4(fmaf(d, xi.x, acc.x), fmaf(d, xi.y, acc.y), fmaf(d, xi.z, acc.z),
                       fmaf(d, xi.w, acc.w));
  } else {
    float acc[kIPT] = {0.f, 0.f, 0.f, 0.f}, dsum[kIPT] = {0.f, 0.f, 0.f, 0.f};
    for (int32_t j = 0; j < W; j += U) {
      int32_t c[U];
      float m[U][kIPT];
      float4 xv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool ok = j + u < W;
        const int64_t p = base + C * (j + u) + r;
        if constexpr (KIND == kStates) {
          const int2 e = ok ? __ldg(a.Lcw + p) : make_int2(rr, 0);
          const int f = ok ? (int)__ldg(a.Lfc + p) : 0;
          c[u] = e.x;
          const float w = __int_as_float(e.y);
#pragma unroll
          for (int jj = 0; jj < kIPT; ++jj) m[u][jj] = f > st[jj] ? w : 0.0f;
        } else {
          c[u] = ok ? __ldg(a.Lcol + p) : rr;
          const float4 w4 = ok ? __ldg(reinterpret_cast<const float4*>(a.Lw + p * a.BS) + q)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
          m[u][0] = w4.x; m[u][1] = w4.y; m[u][2] = w4.z; m[u][3] = w4.w;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        xv[u] = j + u < W ? X[(int64_t)c[u] * TPR + q] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int jj = 0; jj < kIPT; ++jj) {
          dsum[jj] += m[u][jj];
          acc[jj] = fmaf(m[u][jj], get4(xv[u], jj), acc[jj]);
        }
    }
    float4 y;
#pragma unroll
    for (int jj = 0; jj < kIPT; ++jj)
      set4(y, jj, dsum[jj] == 0.0f ? get4(xi, jj) : fmaf(dsum[jj], get4(xi, jj), -acc[jj]));
    return y;
  }
}

// (L_b x)_i in FP64 (the residual of a reliable update)
template <int KIND>
__device__ __forceinline__ void l_row64(const BatchArgs& a, int64_t s, int r, int q,
                                        int32_t row, const int (&st)[kIPT],
                                        const double* __restrict__ X, double (&y)[kIPT]) {
  const int C = a.C, BS = a.BS;
  const int32_t base = a.Lsptr[s];
  const int32_t W = (a.Lsptr[s + 1] - base) / C;
  const int32_t rr = row >= 0 ? row : 0;
  const double* xi = X + (int64_t)rr * BS + kIPT * q;
  double acc[kIPT] = {0.0, 0.0, 0.0, 0.0}, dsum[kIPT] = {0.0, 0.0, 0.0, 0.0};
  for (int32_t j = 0; j < W; ++j) {
    const int64_t p = base + C * j + r;
    int32_t c;
    double m[kIPT];
    if constexpr (KIND == kFields) {
      c = __ldg(a.Lcol + p);
#pragma unroll
      for (int jj = 0; jj < kIPT; ++jj) m[jj] = __ldg(a.L64 + p * BS + kIPT * q + jj);
    } else {
      c = __ldg(a.Lcw + p).x;
      const double w = __ldg(a.L64 + p);
      const int f = KIND == kStates ? (int)__ldg(a.Lfc + p) : 0;
#pragma unroll
      for (int jj = 0; jj < kIPT; ++jj) m[jj] = (KIND == kSets || f > st[jj]) ? w : 0.0;
    }
    const double2 x01 = *reinterpret_cast<const double2*>(X + (int64_t)c * BS + kIPT * q);
    const double2 x23 = *reinterpret_cast<const double2*>(X + (int64_t)c * BS + kIPT * q + 2);
    const double xc[kIPT] = {x01.x, x01.y, x23.x, x23.y};
#pragma unroll
    for (int jj = 0; jj < kIPT; ++jj) {
      dsum[jj] += m[jj];
      acc[jj] = fma(m[jj], xc[jj], acc[jj]);
    }
  }
  if constexpr (KIND == kSets) {
    const double d = a.d64[rr];
#pragma unroll
    for (int jj = 0; jj < kIPT; ++jj) y[jj] = fma(d, xi[jj], acc[jj]);
  } else {
#pragma unroll
    for (int jj = 0; jj < kIPT; ++jj)
      y[jj] = dsum[jj] == 0.0 ? xi[jj] : fma(dsum[jj], xi[jj], -acc[jj]);
  }
}

// One FSAI half (h = 0: G, h = 1: G^T) for the four instances of lane (r, q)
template <int U>
__device__ __forceinline__ float4 g_row(const BatchArgs& a, int h, int64_t s, int r, int q,
                                        int32_t row, const float4* __restrict__ X) {
  const int C = a.C, TPR = a.TPR;
  const int32_t base = a.Gsptr[h][s];
  const int32_t W = (a.Gsptr[h][s + 1] - base) / C;
  const int32_t rr = row >= 0 ? row : 0;
  const int32_t* __restrict__ col = a.Gcol[h];
  const __nv_bfloat16* __restrict__ gv = a.Gv[h];
  const __nv_bfloat16* __restrict__ gb = a.Gb[h];
  float acc[kIPT] = {0.f, 0.f, 0.f, 0.f};
  for (int32_t j = 0; j < W; j += U) {
    int32_t c[U];
    float g[U][kIPT];
    float4 xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = j + u < W;
      const int64_t p = base + C * (j + u) + r;
      c[u] = ok ? __ldg(col + p) : rr;
      if (!ok) {
#pragma unroll
        for (int jj = 0; jj < kIPT; ++jj) g[u][jj] = 0.0f;
      } else if (gb) {
        const uint2 raw = __ldg(reinterpret_cast<const uint2*>(gb + p * a.BS) + q);
        const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&raw.x);
        const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&raw.y);
        g[u][0] = __low2float(lo); g[u][1] = __high2float(lo);
        g[u][2] = __low2float(hi); g[u][3] = __high2float(hi);
      } else {
        const float gs = __bfloat162float(gv[p]);
#pragma unroll
        for (int jj = 0; jj < kIPT; ++jj) g[u][jj] = gs;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      xv[u] = j + u < W ? X[(int64_t)c[u] * TPR + q] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int jj = 0; jj < kIPT; ++jj) acc[jj] = fmaf(g[u][jj], get4(xv[u], jj), acc[jj]);
  }
  return make_float4(acc[0], acc[1], acc[2], acc[3]);
}

// Dot-product accumulator: FP32 products folded into FP64 every 16 terms,
// so the narrow FP64 pipe sees one add per 16 elements.
struct Acc2 {
  double d = 0.0;
  float f = 0.0f;
  int c = 0;
  __device__ __forceinline__ void add(float x, float y) {
    f = fmaf(x, y, f);
    if (++c == 16) { d += (double)f; f = 0.0f; c = 0; }
  }
  __device__ __forceinline__ double get() const { return d + (double)f; }
};

// The vector phases run in element order: element e of a [n][BS] vector
// seen as float4s belongs to quad e % TPR, and with a stride that is a
// multiple of 1024 every thread stays on its own quad q = lane % TPR.
template <int KIND, int U>
__global__ void __launch_bounds__(kBBlock, 1)
pcg_batched_persistent(BatchArgs a) {
  // barrier test: bar[3] != 0 withholds the last block, so the others'
  // first barrier wait runs out (DEC_ERR_TIMEOUT)
  if (*(volatile unsigned*)(a.bar + 3) && blockIdx.x == gridDim.x - 1) return;
  __shared__ BState S;
  __shared__ double shw[kBWarps][kBMax];
  const int BS = a.BS, TPR = a.TPR, C = a.C;
  const int64_t n = a.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = lane / TPR, q = lane % TPR;            // row slot, instance quad
  const int64_t nq = n * TPR;                          // float4 elements of a vector
  const int64_t e0 = (int64_t)blockIdx.x * kBBlock + threadIdx.x;
  const int64_t estep = (int64_t)gridDim.x * kBBlock;
  int st[kIPT];
#pragma unroll
  for (int j = 0; j < kIPT; ++j) st[j] = kIPT * q + j;
  int* err = a.status;
  int parity = 0;
  float4* X = reinterpret_cast<float4*>(a.x);
  float4* R = reinterpret_cast<float4*>(a.r);
  float4* Z = reinterpret_cast<float4*>(a.z);
  float4* Pv = reinterpret_cast<float4*>(a.p);
  float4* Q = reinterpret_cast<float4*>(a.q);
  float4* T = reinterpret_cast<float4*>(a.t);
  auto act = [&](const int* flags, int j) { return flags[kIPT * q + j] != 0; };
  auto any4 = [&](const int* flags) {
    return flags[kIPT * q] | flags[kIPT * q + 1] | flags[kIPT * q + 2] | flags[kIPT * q + 3];
  };
  // the slices of this block: one per warp in each window it owns
  auto windows = [&](const int32_t* perm, auto&& body) {
    for (int64_t win = blockIdx.x; win < a.nwin; win += gridDim.x) {
      const int64_t s = win * kBWarps + warp;
      body(s, __ldg(perm + s * C + r));
    }
  };
  auto vec4 = [&](const float* v) {
    float4 o;
#pragma unroll
    for (int j = 0; j < kIPT; ++j) set4(o, j, v[kIPT * q + j]);
    return o;
  };

  // ---- start: x64 = 0, r64 = b, r = (float) b, x = p = 0, |b|^2 per
  // instance; a warm start keeps x64 and forms r64 = b - L x64 instead
  {
    double v[kIPT] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t e = e0; e < nq; e += estep) {
      float4 rf;
#pragma unroll
      for (int j = 0; j < kIPT; ++j) {
        const double bi = a.bvec[e * kIPT + j];
        if (!a.warm) {
          a.x64[e * kIPT + j] = 0.0;
          a.r64[e * kIPT + j] = bi;
        }
        set4(rf, j, (float)bi);
        v[j] = fma(bi, bi, v[j]);
      }
      if (!a.warm) R[e] = rf;
      X[e] = make_float4(0.f, 0.f, 0.f, 0.f);
      Pv[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (!breduce(v, a, parity, S, shw, err)) return;
  }
  if (threadIdx.x < BS) S.bnorm2[threadIdx.x] = S.red[threadIdx.x];
  __syncthreads();
  if (a.warm) {
    double v[kIPT] = {0.0, 0.0, 0.0, 0.0};
    windows(a.Lperm, [&](int64_t s, int32_t row) {
      double y[kIPT];
      l_row64<KIND>(a, s, r, q, row, st, a.x64, y);
      if (row < 0) return;
      float4 rf;
#pragma unroll
      for (int j = 0; j < kIPT; ++j) {
        const int64_t e = (int64_t)row * BS + kIPT * q + j;
        const double ri = a.bvec[e] - y[j];
        a.r64[e] = ri;
        set4(rf, j, (float)ri);
        v[j] = fma(ri, ri, v[j]);
      }
      R[(int64_t)row * TPR + q] = rf;
    });
    if (!breduce(v, a, parity, S, shw, err)) return;
  }
  if (threadIdx.x < BS) {
    const int i = threadIdx.x;
    const double rr = S.red[i];         // |r0|^2 (= |b|^2 from x = 0)
    S.best[i] = rr;
    S.tol2[i] = a.seg2 * rr;
    a.result[i] = rr;
    S.active[i] = (i < a.B && S.bnorm2[i] > 0.0 && rr > a.rtol2 * S.bnorm2[i]) ? 1 : 0;
    S.iterating[i] = S.active[i];
    S.restart[i] = 1;
    S.stall[i] = 0;
    S.iters[i] = 0;
    S.rz[i] = 0.0;
  }
  __syncthreads();

  // z = M r = G^T (G r) on the instances in `flags`, with r.z per instance
  auto apply_precond = [&](const int* flags) -> bool {
    if (any4(flags))
      windows(a.Gperm[0], [&](int64_t s, int32_t row) {
        const float4 y = g_row<U>(a, 0, s, r, q, row, R);
        if (row >= 0) T[(int64_t)row * TPR + q] = y;
      });
    if (!bgrid_sync(a.bar, err)) return false;
    Acc2 acc[kIPT];
    if (any4(flags))
      windows(a.Gperm[1], [&](int64_t s, int32_t row) {
        const float4 zi = g_row<U>(a, 1, s, r, q, row, T);
        if (row < 0) return;
        Z[(int64_t)row * TPR + q] = zi;
        const float4 ri = R[(int64_t)row * TPR + q];
#pragma unroll
        for (int j = 0; j < kIPT; ++j) acc[j].add(get4(ri, j), get4(zi, j));
      });
    double v[kIPT];
#pragma unroll
    for (int j = 0; j < kIPT; ++j) v[j] = acc[j].get();
    return breduce(v, a, parity, S, shw, err);
  };

  for (;;) {
    // ---- segment start for the active instances: z = M r, p = z + beta p
    if (!apply_precond(S.active)) return;
    if (threadIdx.x < BS) {
      const int i = threadIdx.x;
      const double rzn = S.red[i];
      S.beta[i] = (S.restart[i] || S.rz[i] == 0.0) ? 0.0f : (float)(rzn / S.rz[i]);
      S.rz[i] = rzn;
      S.iterating[i] = S.active[i];
    }
    __syncthreads();
    if (any4(S.active)) {
      const float4 bt = vec4(S.beta);
      for (int64_t e = e0; e < nq; e += estep) {
        const float4 zv = Z[e], pv = Pv[e];
        Pv[e] = make_float4(fmaf(bt.x, pv.x, zv.x), fmaf(bt.y, pv.y, zv.y),
                            fmaf(bt.z, pv.z, zv.z), fmaf(bt.w, pv.w, zv.w));
      }
    }
    if (!bgrid_sync(a.bar, err)) return;

    // ---- FP32 iterations until every working instance is frozen
    for (;;) {
      {
        Acc2 acc[kIPT];
        if (any4(S.iterating))
          windows(a.Lperm, [&](int64_t s, int32_t row) {
            const float4 qi = l_row<KIND, U>(a, s, r, q, row, st, Pv);
            if (row < 0) return;
            Q[(int64_t)row * TPR + q] = qi;
            const float4 pi = Pv[(int64_t)row * TPR + q];
#pragma unroll
            for (int j = 0; j < kIPT; ++j) acc[j].add(get4(pi, j), get4(qi, j));
          });
        double v[kIPT];
#pragma unroll
        for (int j = 0; j < kIPT; ++j) v[j] = acc[j].get();
        if (!breduce(v, a, parity, S, shw, err)) return;
      }
      if (threadIdx.x < BS) {
        const int i = threadIdx.x;
        const double pq = S.red[i];
        if (S.iterating[i] && (!(pq > 0.0) || !isfinite(pq))) {
          S.iterating[i] = 0;             // breakdown: freeze and restart
          S.restart[i] = 1;
        }
        S.alpha[i] = S.iterating[i] ? (float)(S.rz[i] / pq) : 0.0f;
      }
      __syncthreads();
      {
        Acc2 acc[kIPT];
        if (any4(S.iterating)) {
          const float4 al = vec4(S.alpha);
          for (int64_t e = e0; e < nq; e += estep) {
            const float4 qv = Q[e], rv = R[e], pv = Pv[e], xv = X[e];
            const float4 rn = make_float4(fmaf(-al.x, qv.x, rv.x), fmaf(-al.y, qv.y, rv.y),
                                          fmaf(-al.z, qv.z, rv.z), fmaf(-al.w, qv.w, rv.w));
            X[e] = make_float4(fmaf(al.x, pv.x, xv.x), fmaf(al.y, pv.y, xv.y),
                               fmaf(al.z, pv.z, xv.z), fmaf(al.w, pv.w, xv.w));
            R[e] = rn;
#pragma unroll
            for (int j = 0; j < kIPT; ++j) acc[j].add(get4(rn, j), get4(rn, j));
          }
        }
        double v[kIPT];
#pragma unroll
        for (int j = 0; j < kIPT; ++j) v[j] = acc[j].get();
        if (!breduce(v, a, parity, S, shw, err)) return;
      }
      if (threadIdx.x < BS) {
        const int i = threadIdx.x;
        if (S.iterating[i]) {
          S.iters[i] += 1;
          const double rr = S.red[i];
          if (rr <= S.tol2[i] || S.iters[i] >= a.max_iter || !isfinite(rr)) S.iterating[i] = 0;
        }
      }
      if (threadIdx.x == 0) {
        int c = 0;
        for (int i = 0; i < BS; ++i) c += S.iterating[i];
        S.count = c;
      }
      __syncthreads();
      if (S.count == 0) break;
      // preconditioner on the iterating instances
      if (!apply_precond(S.iterating)) return;
      if (threadIdx.x < BS) {
        const int i = threadIdx.x;
        if (S.iterating[i]) {
          S.beta[i] = (float)(S.red[i] / S.rz[i]);
          S.rz[i] = S.red[i];
        }
      }
      __syncthreads();
      if (any4(S.iterating)) {
        const float4 bt = vec4(S.beta);
        bool on[kIPT];
#pragma unroll
        for (int j = 0; j < kIPT; ++j) on[j] = act(S.iterating, j);
        for (int64_t e = e0; e < nq; e += estep) {
          const float4 zv = Z[e];
          float4 pv = Pv[e];
          if (on[0]) pv.x = fmaf(bt.x, pv.x, zv.x);
          if (on[1]) pv.y = fmaf(bt.y, pv.y, zv.y);
          if (on[2]) pv.z = fmaf(bt.z, pv.z, zv.z);
          if (on[3]) pv.w = fmaf(bt.w, pv.w, zv.w);
          Pv[e] = pv;
        }
      }
      if (!bgrid_sync(a.bar, err)) return;
    }

    // ---- reliable update of the active instances
    if (any4(S.active))
      for (int64_t e = e0; e < nq; e += estep) {
        const float4 xv = X[e];
#pragma unroll
        for (int j = 0; j < kIPT; ++j) a.x64[e * kIPT + j] += (double)get4(xv, j);
        X[e] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    if (!bgrid_sync(a.bar, err)) return;
    {
      double v[kIPT] = {0.0, 0.0, 0.0, 0.0};
      if (any4(S.active))
        windows(a.Lperm, [&](int64_t s, int32_t row) {
          double y[kIPT];
          l_row64<KIND>(a, s, r, q, row, st, a.x64, y);
          if (row < 0) return;
          float4 rf;
#pragma unroll
          for (int j = 0; j < kIPT; ++j) {
            const int64_t e = (int64_t)row * BS + kIPT * q + j;
            const double ri = a.bvec[e] - y[j];
            a.r64[e] = ri;
            set4(rf, j, (float)ri);
            v[j] = fma(ri, ri, v[j]);
          }
          R[(int64_t)row * TPR + q] = rf;
        });
      if (!breduce(v, a, parity, S, shw, err)) return;
    }
    if (threadIdx.x < BS) {
      const int i = threadIdx.x;
      if (S.active[i]) {
        const double rr = S.red[i];
        a.result[i] = rr;
        if (rr <= a.rtol2 * S.bnorm2[i] || S.iters[i] >= a.max_iter) {
          S.active[i] = 0;
        } else {
          if (rr < 0.5 * S.best[i]) { S.best[i] = rr; S.stall[i] = 0; S.restart[i] = 0; }
          else { S.stall[i] += 1; S.restart[i] = 1; }
          if (S.stall[i] >= 4) S.active[i] = 0;
          S.tol2[i] = a.seg2 * rr;
        }
      }
    }
    if (threadIdx.x == 0) {
      int c = 0;
      for (int i = 0; i < BS; ++i) c += S.active[i];
      S.count = c;
    }
    __syncthreads();
    if (S.count == 0) break;
  }
  if (blockIdx.x == 0 && threadIdx.x < BS) {
    a.iters[threadIdx.x] = S.iters[threadIdx.x];
    a.result[BS + threadIdx.x] = S.bnorm2[threadIdx.x];
  }
}

// ------------------------------------------------------------ set-up
// *1 of CSR entry k in instance b (0 on the diagonal): Dirichlet sets use
// the cracks of the single state, crack states state b, fields field b's *1
// with the cracks of the single state.
struct EntryWeights {
  const int32_t* eid;
  const double* w;          // [ne] or [n_fields][ne]
  const uint8_t* fc;        // first crack state per edge
  int64_t ne;
  int kind;
  __device__ __forceinline__ double operator()(int32_t k, int b) const {
    const int32_t e = eid[k];
    if (e < 0) return 0.0;
    const int f = (int)fc[e];
    if (kind == kStates) return f > b ? w[e] : 0.0;
    if (kind == kFields) return f > 0 ? w[(int64_t)b * ne + e] : 0.0;
    return f > 0 ? w[e] : 0.0;
  }
};

// Per-instance FSAI factors for the batched solve (same definition as the
// single-instance factor: row i solves L_b[P_i, P_i] g = e_i and stores
// g / sqrt(g_i)), computed in FP32 from the edge form of L_b and stored in
// BF16 in CSR order with the instances contiguous: entries with col <= row
// hold G[row][col], entries with col > row G[col][row].  A group of BS
// threads handles one row, thread b instance b, each with the packed lower
// triangle of its block in shared memory (k <= kBFsaiMax).  Longer rows
// (about 3 % of the rows at a limit of 12, which lets two blocks share an
// SM) keep the shared factor g0 (the uncracked operator's for crack states,
// field 0's for fields).
#ifndef DEC_BFSAI_MAX
#define DEC_BFSAI_MAX 12
#endif
constexpr int kBFsaiMax = DEC_BFSAI_MAX;
constexpr int kBFsaiTpb = 256;
constexpr int kBPacked = kBFsaiMax * (kBFsaiMax + 1) / 2;

__device__ __forceinline__ int btri(int r, int c) { return r * (r + 1) / 2 + c; }

__global__ void __launch_bounds__(kBFsaiTpb)
batch_fsai_kernel(int64_t n, int BS, int B, EntryWeights wt, const int32_t* __restrict__ rowptr,
                  const int32_t* __restrict__ col, const int32_t* __restrict__ dpos,
                  const int32_t* __restrict__ pos_up, const uint8_t* __restrict__ tag,
                  const double* __restrict__ g0, __nv_bfloat16* __restrict__ gb) {
  extern __shared__ float bsm[];
  float* A = bsm + threadIdx.x;                                  // stride kBFsaiTpb
  int32_t* P = reinterpret_cast<int32_t*>(bsm + kBPacked * kBFsaiTpb) + threadIdx.x;
  const int stride = kBFsaiTpb;
  const int b = threadIdx.x % BS;
  const int inst = b < B ? b : 0;           // padding instances copy instance 0
  const int rpb = kBFsaiTpb / BS;
  for (int64_t i = (int64_t)blockIdx.x * rpb + threadIdx.x / BS; i < n;
       i += (int64_t)gridDim.x * rpb) {
    const int32_t k0 = rowptr[i], kd = dpos[i];
    const int k = kd - k0 + 1;
    if (k > kBFsaiMax) {   // this row's lower part and its transposed slots
      for (int32_t kk = k0; kk <= kd; ++kk) {
        const __nv_bfloat16 g = __float2bfloat16_rn((float)g0[kk]);
        gb[(int64_t)kk * BS + b] = g;
        if (kk < kd) gb[(int64_t)pos_up[wt.eid[kk]] * BS + b] = g;
      }
      continue;
    }
    for (int qq = 0; qq < k; ++qq) P[qq * stride] = col[k0 + qq];
    float dmax = 0.0f;
    bool ok = true;
    for (int pass = 0; pass < 2; ++pass) {
      // gather L_b[P, P] (edge form; Dirichlet rows/columns eliminated),
      // with a shift of 1e-5 max(diag) on the second pass
      const float shift = pass == 0 ? 0.0f : 1e-5f * dmax;
      for (int qq = 0; qq < k; ++qq) {
        const int32_t rw = P[qq * stride];
        for (int c = 0; c < qq; ++c) A[btri(qq, c) * stride] = 0.0f;
        if (tag[rw] == DEC_NODE_DIRICHLET) {
          A[btri(qq, qq) * stride] = 1.0f + shift;
          if (pass == 0) dmax = fmaxf(dmax, 1.0f);
          continue;
        }
        float dsum = 0.0f;
        int c = 0;
        for (int32_t kk = rowptr[rw]; kk < rowptr[rw + 1]; ++kk) {
          const float m = (float)wt(kk, inst);
          dsum += m;
          const int32_t cc = col[kk];
          if (kk < dpos[rw]) {            // lower part of row rw: columns < rw
            while (c < qq && P[c * stride] < cc) ++c;
            if (c < qq && P[c * stride] == cc && tag[cc] != DEC_NODE_DIRICHLET)
              A[btri(qq, c) * stride] = -m;
          }
        }
        A[btri(qq, qq) * stride] = (dsum == 0.0f ? 1.0f : dsum) + shift;
        if (pass == 0) dmax = fmaxf(dmax, A[btri(qq, qq) * stride]);
      }
      // Cholesky in place; a pivot <= 1e-6 max(diag) marks a singular block
      ok = true;
      for (int c = 0; c < k && ok; ++c) {
        const float d = A[btri(c, c) * stride];
        if (!(d > (pass == 0 ? 1e-6f * dmax : 0.0f))) { ok = false; break; }
        const float lc = sqrtf(d), inv = 1.0f / lc;
        A[btri(c, c) * stride] = lc;
        for (int rw = c + 1; rw < k; ++rw) A[btri(rw, c) * stride] *= inv;
        for (int rw = c + 1; rw < k; ++rw) {
          const float lrc = A[btri(rw, c) * stride];
          for (int qq = c + 1; qq <= rw; ++qq)
            A[btri(rw, qq) * stride] -= lrc * A[btri(qq, c) * stride];
        }
      }
      if (ok) break;
    }
    // C^T g = e_k, g_j over the used diagonal slot
    for (int j = k - 1; j >= 0; --j) {
      float sum = (j == k - 1) ? 1.0f : 0.0f;
      for (int rw = j + 1; rw < k; ++rw) sum -= A[btri(rw, j) * stride] * A[btri(rw, rw) * stride];
      A[btri(j, j) * stride] = ok ? sum / A[btri(j, j) * stride] : 0.0f;
    }
    for (int qq = 0; qq < k; ++qq) {
      const __nv_bfloat16 gq = ok ? __float2bfloat16_rn(A[btri(qq, qq) * stride])
                                  : __float2bfloat16_rn((float)g0[k0 + qq]);
      gb[(int64_t)(k0 + qq) * BS + b] = gq;
      if (qq < k - 1) gb[(int64_t)pos_up[wt.eid[k0 + qq]] * BS + b] = gq;
    }
  }
}

// Morton key of a node: 21 bits per coordinate of its position in the
// bounding box, bits interleaved (x lowest)
__device__ __forceinline__ uint64_t spread21(uint64_t v) {
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

__global__ void morton_keys_kernel(int64_t n, const double* __restrict__ xyz, double3 lo,
                                   double3 scale, uint64_t* __restrict__ key,
                                   uint32_t* __restrict__ val) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double fx = (xyz[3 * i] - lo.x) * scale.x;
    const double fy = (xyz[3 * i + 1] - lo.y) * scale.y;
    const double fz = (xyz[3 * i + 2] - lo.z) * scale.z;
    const uint64_t ix = (uint64_t)fmin(fmax(fx, 0.0), 2097151.0);
    const uint64_t iy = (uint64_t)fmin(fmax(fy, 0.0), 2097151.0);
    const uint64_t iz = (uint64_t)fmin(fmax(fz, 0.0), 2097151.0);
    key[i] = spread21(ix) | (spread21(iy) << 1) | (spread21(iz) << 2);
    val[i] = (uint32_t)i;
  }
}

// rank[order[p]] = p
__global__ void invert_order_kernel(int64_t n, const int32_t* __restrict__ order,
                                    int32_t* __restrict__ rank) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x)
    rank[order[p]] = (int32_t)p;
}

// a sliced layout built over node ids, renumbered to Morton positions
__global__ void renumber_layout_kernel(int64_t slots, int64_t total,
                                       const int32_t* __restrict__ rank,
                                       int32_t* __restrict__ perm, int32_t* __restrict__ col) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < slots || p < total;
       p += (int64_t)gridDim.x * blockDim.x) {
    if (p < slots && perm[p] >= 0) perm[p] = rank[perm[p]];
    if (p < total) col[p] = rank[col[p]];
  }
}

// bounding box of the nodes: out = (min x, min y, min z, max x, max y, max z)
__global__ void bbox_kernel(int64_t n, const double* __restrict__ xyz, double* __restrict__ out) {
  __shared__ double sh[6][256];
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
    for (int d = 0; d < 3; ++d) {
      lo[d] = fmin(lo[d], xyz[3 * i + d]);
      hi[d] = fmax(hi[d], xyz[3 * i + d]);
    }
  for (int d = 0; d < 3; ++d) {
    sh[d][threadIdx.x] = lo[d];
    sh[3 + d][threadIdx.x] = hi[d];
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = sh[threadIdx.x][0];
    for (int j = 1; j < (int)blockDim.x; ++j)
      v = threadIdx.x < 3 ? fmin(v, sh[threadIdx.x][j]) : fmax(v, sh[threadIdx.x][j]);
    out[threadIdx.x] = v;
  }
}

// Values of the batched L in its sliced layout, from CSR entry k.
__global__ void batch_l_values_kernel(int64_t nnz, int kind, int BS, int B,
                                      const int32_t* __restrict__ pos, EntryWeights wt,
                                      const double* __restrict__ val64, int2* __restrict__ cw,
                                      uint8_t* __restrict__ lfc, float* __restrict__ lw,
                                      double* __restrict__ l64) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = pos[k];
    if (p < 0) continue;
    if (kind == kSets) {
      cw[p].y = __float_as_int((float)val64[k]);
      l64[p] = val64[k];
    } else if (kind == kStates) {
      const int32_t e = wt.eid[k];
      cw[p].y = __float_as_int((float)wt.w[e]);
      l64[p] = wt.w[e];
      lfc[p] = wt.fc[e];
    } else {
      for (int b = 0; b < BS; ++b) {
        const double we = b < B ? wt(k, b) : 0.0;
        lw[(int64_t)p * BS + b] = (float)we;
        l64[(int64_t)p * BS + b] = we;
      }
    }
  }
}

// (column, 0) for every slot of the sliced L (padding included)
__global__ void batch_cw_init_kernel(int64_t total, const int32_t* __restrict__ col,
                                     int2* __restrict__ cw) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total;
       p += (int64_t)gridDim.x * blockDim.x)
    cw[p] = make_int2(col[p], 0);
}

__global__ void batch_diag_kernel(int64_t n, const int32_t* __restrict__ dpos,
                                  const int32_t* __restrict__ rank,
                                  const double* __restrict__ val64, float* __restrict__ d32,
                                  double* __restrict__ d64) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = val64[dpos[i]];
    d32[rank[i]] = (float)d;
    d64[rank[i]] = d;
  }
}

// shared factor halves in their sliced layouts (CSR layout of g64: lower
// slots G[row][col], upper slots G[col][row])
__global__ void batch_g_values_kernel(int64_t nnz, const int32_t* __restrict__ pos_lo,
                                      const int32_t* __restrict__ pos_hi,
                                      const double* __restrict__ g64,
                                      __nv_bfloat16* __restrict__ glo,
                                      __nv_bfloat16* __restrict__ ghi) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x) {
    const __nv_bfloat16 g = __float2bfloat16_rn((float)g64[k]);
    if (pos_lo[k] >= 0) glo[pos_lo[k]] = g;
    if (pos_hi[k] >= 0) ghi[pos_hi[k]] = g;
  }
}

// per-instance factor halves from the CSR-order per-instance factor
__global__ void batch_gb_scatter_kernel(int64_t nnz, int BS, const int32_t* __restrict__ pos_lo,
                                        const int32_t* __restrict__ pos_hi,
                                        const __nv_bfloat16* __restrict__ gb,
                                        __nv_bfloat16* __restrict__ glo,
                                        __nv_bfloat16* __restrict__ ghi) {
  const int64_t total = nnz * BS;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t / BS;
    const int b = (int)(t % BS);
    const __nv_bfloat16 g = gb[t];
    if (pos_lo[k] >= 0) glo[(int64_t)pos_lo[k] * BS + b] = g;
    if (pos_hi[k] >= 0) ghi[(int64_t)pos_hi[k] * BS + b] = g;
  }
}

// right-hand sides b[i][inst] = sum over Dirichlet neighbours j of
// w_ij(inst) T0_j (0 on Dirichlet rows and on rows all of whose weights are
// zero in that instance), the node form of Eq. 12
__global__ void batch_rhs_kernel(int64_t n, int B, int BS, int sets, EntryWeights wt,
                                 const int32_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ col,
                                 const int32_t* __restrict__ dpos,
                                 const uint8_t* __restrict__ tag,
                                 const int32_t* __restrict__ rank,
                                 const double* __restrict__ T0, double* __restrict__ bvec) {
  const int64_t ne = n * BS;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / BS;
    const int inst = (int)(e % BS);
    double bi = 0.0;
    if (inst < B && tag[i] != DEC_NODE_DIRICHLET) {
      const double* t0 = T0 + (sets ? (int64_t)inst * n : 0);
      double dsum = 0.0;
      for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        if (k == dpos[i]) continue;
        const double m = wt(k, inst);
        dsum += m;
        if (tag[col[k]] == DEC_NODE_DIRICHLET) bi += m * t0[col[k]];
      }
      if (dsum == 0.0) bi = 0.0;
    }
    bvec[(int64_t)rank[i] * BS + inst] = bi;
  }
}

// rhs of every instance in the per-instance layout b[inst][i] (getters)
__global__ void batch_rhs_unpack_kernel(int64_t n, int B, int BS,
                                        const int32_t* __restrict__ rank,
                                        const double* __restrict__ bb, double* __restrict__ b) {
  const int64_t total = n * B;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t inst = k / n, i = k % n;
    b[k] = bb[(int64_t)rank[i] * BS + inst];
  }
}

// u[inst][i] = x64[rank i][inst]
__global__ void batch_unpack_kernel(int64_t n, int B, int BS, const int32_t* __restrict__ rank,
                                    const double* __restrict__ x64, double* __restrict__ u) {
  const int64_t total = n * B;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t inst = k / n, i = k % n;
    u[k] = x64[(int64_t)rank[i] * BS + inst];
  }
}

int batch_stride(int B) {
  int bs = 8;
  while (bs < B) bs <<= 1;
  return bs;
}

static unsigned grid_for_work(const dec_ctx* ctx, int64_t work) {
  return (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((work + 255) / 256, (int64_t)ctx->num_sms * 16));
}

// Morton order of the nodes (the windows of the batched layouts)
static dec_status build_morton(dec_ctx* ctx) {
  const int64_t n = ctx->n;
  cudaStream_t s = ctx->stream;
  DEC_TRY(ctx->kpartial.ensure(8));
  bbox_kernel<<<1, 256, 0, s>>>(n, ctx->xyz.p, ctx->kpartial.p);
  double bb[6];
  DEC_TRY(cudaMemcpyAsync(bb, ctx->kpartial.p, sizeof(bb), cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaStreamSynchronize(s));
  const double3 lo = make_double3(bb[0], bb[1], bb[2]);
  const double span[3] = {bb[3] - bb[0], bb[4] - bb[1], bb[5] - bb[2]};
  const double3 sc = make_double3(span[0] > 0 ? 2097151.0 / span[0] : 0.0,
                                  span[1] > 0 ? 2097151.0 / span[1] : 0.0,
                                  span[2] > 0 ? 2097151.0 / span[2] : 0.0);
  DEC_TRY(ctx->key_a.ensure(n));
  DEC_TRY(ctx->key_b.ensure(n));
  DEC_TRY(ctx->val_a.ensure(n));
  DEC_TRY(ctx->val_b.ensure(n));
  morton_keys_kernel<<<grid_for_work(ctx, n), 256, 0, s>>>(n, ctx->xyz.p, lo, sc, ctx->key_a.p,
                                                           ctx->val_a.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 2;
  bool alt = false;
  DEC_TRY_STATUS(radix_sort_pairs(ctx, ctx->key_a.p, ctx->val_a.p, ctx->key_b.p, ctx->val_b.p,
                                  n, 63, &alt));
  DEC_TRY(ctx->morton.ensure(n));
  DEC_TRY(ctx->mrank.ensure(n));
  DEC_TRY(cudaMemcpyAsync(ctx->morton.p, alt ? ctx->val_b.p : ctx->val_a.p,
                          sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  invert_order_kernel<<<grid_for_work(ctx, n), 256, 0, s>>>(n, ctx->morton.p, ctx->mrank.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 1;
  return DEC_OK;
}

// Values of the sliced layouts (L, the factors) and b[n][BS].
static dec_status batch_values(dec_ctx* ctx) {
  const int64_t n = ctx->n, nnz = ctx->nnz;
  cudaStream_t s = ctx->stream;
  const int B = ctx->B, BS = batch_stride(B);
  const int kind = ctx->batch_kind;
  const EntryWeights wt{ctx->eid.p, ctx->w.p, ctx->first_cut.p, ctx->ne, kind};
  const int64_t tL = ctx->bL.total, tlo = ctx->bGlo.total, tup = ctx->bGup.total;
  // L values
  if (kind == kFields) {
    DEC_TRY(ctx->bLw.ensure((size_t)tL * BS));
    DEC_TRY(ctx->bL64.ensure((size_t)tL * BS));
    DEC_TRY(cudaMemsetAsync(ctx->bLw.p, 0, sizeof(float) * tL * BS, s));
    DEC_TRY(cudaMemsetAsync(ctx->bL64.p, 0, sizeof(double) * tL * BS, s));
  } else {
    DEC_TRY(ctx->bLcw.ensure(tL));
    DEC_TRY(ctx->bL64.ensure(tL));
    DEC_TRY(cudaMemsetAsync(ctx->bL64.p, 0, sizeof(double) * tL, s));
    batch_cw_init_kernel<<<grid_for_work(ctx, tL), 256, 0, s>>>(tL, ctx->bL.col.p, ctx->bLcw.p);
    ctx->launches += 1;
    if (kind == kStates) {
      DEC_TRY(ctx->bLfc.ensure(tL));
      DEC_TRY(cudaMemsetAsync(ctx->bLfc.p, 0, tL, s));
    }
  }
  batch_l_values_kernel<<<grid_for_work(ctx, nnz), 256, 0, s>>>(
      nnz, kind, BS, B, ctx->bL.pos.p, wt, ctx->val64.p, ctx->bLcw.p, ctx->bLfc.p, ctx->bLw.p,
      ctx->bL64.p);
  ctx->launches += 1;
  if (kind == kSets) {
    DEC_TRY(ctx->bd32.ensure(n));
    DEC_TRY(ctx->bd64.ensure(n));
    batch_diag_kernel<<<grid_for_work(ctx, n), 256, 0, s>>>(n, ctx->dpos.p, ctx->mrank.p,
                                                            ctx->val64.p, ctx->bd32.p,
                                                            ctx->bd64.p);
    ctx->launches += 1;
  }
  // shared factor halves
  DEC_TRY(ctx->bGlo16.ensure(tlo));
  DEC_TRY(ctx->bGup16.ensure(tup));
  DEC_TRY(cudaMemsetAsync(ctx->bGlo16.p, 0, sizeof(__nv_bfloat16) * tlo, s));
  DEC_TRY(cudaMemsetAsync(ctx->bGup16.p, 0, sizeof(__nv_bfloat16) * tup, s));
  batch_g_values_kernel<<<grid_for_work(ctx, nnz), 256, 0, s>>>(
      nnz, ctx->bGlo.pos.p, ctx->bGup.pos.p, ctx->g64.p, ctx->bGlo16.p, ctx->bGup16.p);
  // right-hand sides
  DEC_TRY(ctx->bb.ensure((size_t)n * BS));
  batch_rhs_kernel<<<grid_for_work(ctx, n * BS), 256, 0, s>>>(
      n, B, BS, ctx->n_sets > 1, wt, ctx->rowptr.p, ctx->col.p, ctx->dpos.p, ctx->tag.p,
      ctx->mrank.p, ctx->T0.p, ctx->bb.p);
  batch_rhs_unpack_kernel<<<grid_for_work(ctx, n * B), 256, 0, s>>>(n, B, BS, ctx->mrank.p,
                                                                   ctx->bb.p, ctx->b.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 3;
  if (kind != kSets) {
    // crack states and fields change L per instance: one FSAI factor each
    DEC_TRY(ctx->bgb.ensure((size_t)nnz * BS));
    const size_t smem = (size_t)kBPacked * kBFsaiTpb * sizeof(float) +
                        (size_t)kBFsaiMax * kBFsaiTpb * sizeof(int32_t);
    DEC_TRY(cudaFuncSetAttribute(batch_fsai_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    const int rpb = kBFsaiTpb / BS;
    const unsigned gf = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((n + rpb - 1) / rpb, (int64_t)ctx->num_sms * 8));
    batch_fsai_kernel<<<gf, kBFsaiTpb, smem, s>>>(n, BS, B, wt, ctx->rowptr.p, ctx->col.p,
                                                  ctx->dpos.p, ctx->pos_up.p, ctx->tag.p,
                                                  ctx->g64.p, ctx->bgb.p);
    DEC_TRY(ctx->bGloB.ensure((size_t)tlo * BS));
    DEC_TRY(ctx->bGupB.ensure((size_t)tup * BS));
    DEC_TRY(cudaMemsetAsync(ctx->bGloB.p, 0, sizeof(__nv_bfloat16) * tlo * BS, s));
    DEC_TRY(cudaMemsetAsync(ctx->bGupB.p, 0, sizeof(__nv_bfloat16) * tup * BS, s));
    batch_gb_scatter_kernel<<<grid_for_work(ctx, nnz * BS), 256, 0, s>>>(
        nnz, BS, ctx->bGlo.pos.p, ctx->bGup.pos.p, ctx->bgb.p, ctx->bGloB.p, ctx->bGupB.p);
    DEC_TRY(cudaGetLastError());
    ctx->launches += 2;
    ctx->batch_per_instance = true;
  } else {
    ctx->batch_per_instance = false;   // Dirichlet sets share L and its factor
  }
  DEC_TRY(cudaGetLastError());
  return DEC_OK;
}

// Build the sliced layouts, their values, the factors and b[n][BS].
dec_status batch_setup(dec_ctx* ctx) {
  const int B = ctx->B, BS = batch_stride(B);
  const int TPR = BS / kIPT, C = 32 / TPR, R = kBBlock / TPR;
  const int kind = ctx->n_fields > 1 ? kFields : (ctx->n_scales > 1 ? kStates : kSets);
  ctx->batch_kind = kind;
  ctx->batch_BS = 0;
  DEC_TRY_STATUS(build_morton(ctx));
  DEC_TRY_STATUS(build_sell(ctx, kind == kSets ? 4 : 3, ctx->bL, C, R, ctx->morton.p));
  DEC_TRY_STATUS(build_sell(ctx, 1, ctx->bGlo, C, R, ctx->morton.p));
  DEC_TRY_STATUS(build_sell(ctx, 2, ctx->bGup, C, R, ctx->morton.p));
  // rows and columns in Morton positions
  for (SellLayout* L : {&ctx->bL, &ctx->bGlo, &ctx->bGup}) {
    const int64_t slots = L->nslices * L->C;
    renumber_layout_kernel<<<grid_for_work(ctx, std::max<int64_t>(slots, L->total)), 256, 0,
                             ctx->stream>>>(slots, L->total, ctx->mrank.p, L->perm.p, L->col.p);
    ctx->launches += 1;
  }
  DEC_TRY(cudaGetLastError());
  DEC_TRY_STATUS(batch_values(ctx));
  ctx->batch_BS = BS;
  return DEC_OK;
}

dec_status batch_refresh_values(dec_ctx* ctx) {
  if (ctx->batch_BS != batch_stride(ctx->B))
    return ctx->fail(DEC_ERR_STATE, "batched values: layouts not built");
  return batch_values(ctx);
}

// Kernel variants: entries per round trip (U) for the context's instance
// kind.  All variants of a kind add a row's entries in the same order, so
// the choice never changes a result.
constexpr int kGatherVariants[] = {2, 4, 8};
constexpr int kNumGatherVariants = 3;

template <int KIND>
static const void* batch_kernel(int v) {
  switch (v) {
    case 0: return (const void*)pcg_batched_persistent<KIND, 2>;
    case 1: return (const void*)pcg_batched_persistent<KIND, 4>;
    default: return (const void*)pcg_batched_persistent<KIND, 8>;
  }
}

dec_status solve_batched(dec_ctx* ctx, double rtol, int max_iter, int* iters,
                         double* relres, bool warm) {
  const int64_t n = ctx->n;
  cudaStream_t s = ctx->stream;
  const int B = ctx->B, BS = batch_stride(B);
  if (B > kBMax) return ctx->fail(DEC_ERR_LIMIT, "batched solve: more than 64 instances");
  if (BS != ctx->batch_BS) return ctx->fail(DEC_ERR_STATE, "batched solve: layouts not built");
  int coop = 0;
  DEC_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device));
  if (!coop) return ctx->fail(DEC_ERR_LIMIT, "batched solve: cooperative launch unavailable");
  const int kind = ctx->batch_kind;
  const void* kern[kNumGatherVariants];
  for (int v = 0; v < kNumGatherVariants; ++v)
    kern[v] = kind == kSets     ? batch_kernel<kSets>(v)
              : kind == kStates ? batch_kernel<kStates>(v)
                                : batch_kernel<kFields>(v);
  bool usable[kNumGatherVariants];
  bool any = false;
  for (int v = 0; v < kNumGatherVariants; ++v) {
    int per_sm = 0;
    DEC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern[v], kBBlock, 0));
    usable[v] = per_sm >= 1;
    any = any || usable[v];
  }
  if (!any) return ctx->fail(DEC_ERR_LIMIT, "batched solve: cooperative launch unavailable");
  const int grid = ctx->num_sms;
  const size_t nv = (size_t)n * BS;
  for (auto* bf : {&ctx->bx64, &ctx->br64}) DEC_TRY(bf->ensure(nv));
  for (auto* bf : {&ctx->bx, &ctx->br, &ctx->bz, &ctx->bp, &ctx->bq, &ctx->bt})
    DEC_TRY(bf->ensure(nv));
  DEC_TRY(ctx->bpartial.ensure((size_t)2 * grid * BS));
  DEC_TRY(ctx->coop.ensure(16 + 3 * kBMax));
  unsigned* bar = reinterpret_cast<unsigned*>(ctx->coop.p);
  int* status = reinterpret_cast<int*>(ctx->coop.p + 2);
  int* its = reinterpret_cast<int*>(ctx->coop.p + 16);
  double* result = reinterpret_cast<double*>(ctx->coop.p + 16 + kBMax / 2);
  BatchArgs a{};
  a.n = n;
  a.B = B;
  a.BS = BS;
  a.TPR = BS / kIPT;
  a.C = 32 / a.TPR;
  a.nwin = (n + ctx->bL.R - 1) / ctx->bL.R;
  a.Lperm = ctx->bL.perm.p;
  a.Lsptr = ctx->bL.sptr.p;
  a.Lcw = ctx->bLcw.p;
  a.Lfc = ctx->bLfc.p;
  a.Lcol = ctx->bL.col.p;
  a.Lw = ctx->bLw.p;
  a.L64 = ctx->bL64.p;
  a.d32 = ctx->bd32.p;
  a.d64 = ctx->bd64.p;
  const SellLayout* GL[2] = {&ctx->bGlo, &ctx->bGup};
  for (int h = 0; h < 2; ++h) {
    a.Gperm[h] = GL[h]->perm.p;
    a.Gsptr[h] = GL[h]->sptr.p;
    a.Gcol[h] = GL[h]->col.p;
  }
  a.Gv[0] = ctx->bGlo16.p;
  a.Gv[1] = ctx->bGup16.p;
  a.Gb[0] = ctx->batch_per_instance ? ctx->bGloB.p : nullptr;
  a.Gb[1] = ctx->batch_per_instance ? ctx->bGupB.p : nullptr;
  a.bvec = ctx->bb.p;
  a.x64 = ctx->bx64.p;
  a.r64 = ctx->br64.p;
  a.x = ctx->bx.p; a.r = ctx->br.p; a.z = ctx->bz.p; a.p = ctx->bp.p;
  a.q = ctx->bq.p; a.t = ctx->bt.p;
  a.partial = ctx->bpartial.p;
  a.bar = bar;
  a.status = status;
  a.iters = its;
  a.result = result;
  a.rtol2 = rtol * rtol;
  a.seg2 = 1e-4;
  a.max_iter = max_iter;
  void* args[] = {&a};
  auto launch = [&](int v, int iters_cap) -> cudaError_t {
    a.max_iter = iters_cap;
    a.warm = 0;
    cudaError_t e = cudaMemsetAsync(ctx->coop.p, 0, sizeof(int64_t) * (16 + 3 * kBMax), s);
    if (e == cudaSuccess) e = write_barrier_test(ctx, bar);
    if (e == cudaSuccess)
      e = cudaLaunchCooperativeKernel(kern[v], dim3(grid), dim3(kBBlock), args, 0, s);
    ctx->launches += 1;
    return e;
  };
  // Autotuner: the first batched solve of a problem size at this instance
  // stride times kTuneIters FP32 iterations of every variant and keeps the
  // fastest.  All variants give bit-identical results.
  int slot = 0;
  while ((8 << slot) < BS) ++slot;
  // the choice is kept for later solves of a problem of the same size (the
  // same mesh uploaded again, as a benchmark or a time loop does)
  const bool same = ctx->batch_tune_key[slot][0] == n && ctx->batch_tune_key[slot][1] == ctx->nnz;
  int v = same ? ctx->batch_variant[slot] - 1 : -1;
  if (v < 0) {
    constexpr int kTuneIters = 8;
    cudaEvent_t e0, e1;
    DEC_TRY(cudaEventCreate(&e0));
    DEC_TRY(cudaEventCreate(&e1));
    float best = 0.0f;
    for (int c = 0; c < kNumGatherVariants; ++c) {
      if (!usable[c]) continue;
      DEC_TRY(cudaEventRecord(e0, s));
      DEC_TRY(launch(c, kTuneIters));
      DEC_TRY(cudaEventRecord(e1, s));
      DEC_TRY(cudaEventSynchronize(e1));
      int hs0 = 0;
      DEC_TRY(cudaMemcpy(&hs0, status, sizeof(int), cudaMemcpyDeviceToHost));
      if (hs0) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return ctx->fail(DEC_ERR_TIMEOUT, "batched solve: a grid barrier timed out");
      }
      float ms = 0.0f;
      DEC_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (v < 0 || ms < best) {
        best = ms;
        v = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->batch_variant[slot] = v + 1;
    ctx->batch_tune_key[slot][0] = n;
    ctx->batch_tune_key[slot][1] = ctx->nnz;
  }
  ctx->batch_variant_used = kGatherVariants[v];
  // device time of the solve's launch (dec_get_batch_kernel_ms)
  cudaEvent_t k0, k1;
  DEC_TRY(cudaEventCreate(&k0));
  DEC_TRY(cudaEventCreate(&k1));
  DEC_TRY(cudaEventRecord(k0, s));
  {
    // the solve's launch (a warm start needs x64 from the last solve; the
    // autotuner's trial launches above start from zero and overwrite it, so
    // a warm start after a tuning run starts from zero too)
    a.max_iter = max_iter;
    a.warm = warm && same ? 1 : 0;
    cudaError_t e = cudaMemsetAsync(ctx->coop.p, 0, sizeof(int64_t) * (16 + 3 * kBMax), s);
    if (e == cudaSuccess) e = write_barrier_test(ctx, bar);
    if (e == cudaSuccess)
      e = cudaLaunchCooperativeKernel(kern[v], dim3(grid), dim3(kBBlock), args, 0, s);
    ctx->launches += 1;
    DEC_TRY(e);
  }
  DEC_TRY(cudaEventRecord(k1, s));
  batch_unpack_kernel<<<grid_for_work(ctx, n * B), 256, 0, s>>>(n, B, BS, ctx->mrank.p,
                                                                ctx->bx64.p, ctx->u.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 1;
  int hs[3], hi[kBMax];
  double hr[2 * kBMax];
  DEC_TRY(cudaMemcpyAsync(hs, status, sizeof(hs), cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaMemcpyAsync(hi, its, sizeof(int) * BS, cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaMemcpyAsync(hr, result, sizeof(double) * 2 * BS, cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaStreamSynchronize(s));
  float kms = 0.0f;
  DEC_TRY(cudaEventElapsedTime(&kms, k0, k1));
  cudaEventDestroy(k0);
  cudaEventDestroy(k1);
  ctx->batch_kernel_ms = kms;
  if (hs[0]) return ctx->fail(DEC_ERR_TIMEOUT, "batched solve: a grid barrier timed out");
  dec_status st = DEC_OK;
  for (int i = 0; i < B; ++i) {
    iters[i] = hi[i];
    relres[i] = hr[BS + i] > 0.0 ? std::sqrt(hr[i] / hr[BS + i]) : 0.0;
    if (relres[i] > rtol && st == DEC_OK)
      st = ctx->fail(DEC_NOT_CONVERGED, "batched solve: an instance did not converge");
  }
  return st;
}

}  // namespace dec
