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
  double* phase;                          // [6] per-phase device time, block 0
  int64_t Ltotal, Gtotal[2];              // entries of the sliced layouts
};

// Bulk prefetch of [p, p + bytes) into L2 by the copy engine (TMA),
// clipped to [lo, hi) and widened to 16-byte boundaries inside it.  A hint:
// nothing waits for it.
__device__ __forceinline__ void l2_prefetch(const void* p, size_t bytes, const void* lo,
                                            const void* hi) {
  uintptr_t a = (uintptr_t)p, e = a + bytes;
  const uintptr_t l = ((uintptr_t)lo + 15) & ~(uintptr_t)15, h = (uintptr_t)hi & ~(uintptr_t)15;
  a &= ~(uintptr_t)15;
  e = (e + 15) & ~(uintptr_t)15;
  if (a < l) a = l;
  if (e > h) e = h;
  if (e <= a) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)(e - a))
               : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

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
// instances 4q..4q+3.  Entries are taken U at a time: their structure
// (coalesced loads), then U independent 16-byte gathers of neighbour rows,
// then the FMAs; the structure of the next U entries is loaded while the
// gathers are in flight.  The gathers go to registers, or (SMEM variants)
// to per-thread shared-memory slots by 16-byte cp.async, which takes no
// registers while in flight.  The slice width is uniform across the warp,
// so the guards never diverge; padding entries carry value 0 and the row's
// own column.

__device__ __forceinline__ float4* gather_slots() {
  extern __shared__ __align__(16) float4 bsm_slots[];
  return bsm_slots + threadIdx.x;
}
__device__ __forceinline__ void gather_async(float4* slot, const float4* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(slot);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void gather_wait() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}
template <int U>
constexpr int gather_smem() { return U * kBBlock * (int)sizeof(float4); }

// Staged variants (Dirichlet sets): every warp streams the structure of its
// slices through a private double buffer in shared memory, K entries of its
// C rows per chunk; the 16-byte cp.async copies of the next chunk (of this
// slice, or of the warp's slice in the block's next window) are in flight
// while the current chunk's gathers run, so a row waits for its structure
// once per slice instead of once per few entries.  A chunk holds K * C * 8
// bytes when L is staged too (an L entry: column and FP32 value), K * C * 6
// when only the FSAI halves are (column and BF16 value).
__device__ __forceinline__ void copy16_async(void* dst, const void* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void copy_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void copy_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
template <int K>
constexpr int stage_smem(int C, int entry_bytes = 8) {
  return 2 * kBWarps * K * C * entry_bytes;
}

// Structure of one L entry: column and its raw weight data (value bits;
// for crack states also the first crack state; for fields the four
// instances' weights).
template <int KIND>
struct LEnt {
  int32_t c;
  float w[KIND == kFields ? kIPT : 1];
  int f;
};
template <int KIND>
__device__ __forceinline__ LEnt<KIND> l_load(const BatchArgs& a, int64_t p, bool ok, int32_t rr,
                                             int q) {
  LEnt<KIND> e;
  e.f = 0;
  if constexpr (KIND == kFields) {
    e.c = ok ? __ldg(a.Lcol + p) : rr;
    const float4 w4 = ok ? __ldg(reinterpret_cast<const float4*>(a.Lw + p * a.BS) + q)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
    e.w[0] = w4.x; e.w[1] = w4.y; e.w[2] = w4.z; e.w[3] = w4.w;
  } else {
    const int2 cw = ok ? __ldg(a.Lcw + p) : make_int2(rr, 0);
    e.c = cw.x;
    e.w[0] = __int_as_float(cw.y);
    if constexpr (KIND == kStates) e.f = ok ? (int)__ldg(a.Lfc + p) : 0;
  }
  return e;
}
// weight of entry e for instance jj of the lane's quad
template <int KIND>
__device__ __forceinline__ float l_weight(const LEnt<KIND>& e, int jj, const int (&st)[kIPT]) {
  if constexpr (KIND == kFields) return e.w[jj];
  else if constexpr (KIND == kStates) return e.f > st[jj] ? e.w[0] : 0.0f;
  else return e.w[0];
}

// (L_b x)_i, FP32, for the four instances of lane (r, q)
template <int KIND, int U, bool SMEM, bool PIPE>
__device__ __forceinline__ float4 l_row(const BatchArgs& a, int32_t base, int32_t W, int r,
                                        int q, int32_t row, const int (&st)[kIPT],
                                        const float4* __restrict__ X) {
  const int C = a.C, TPR = a.TPR;
  const int32_t rr = row >= 0 ? row : 0;
  const float4 xi = X[(int64_t)rr * TPR + q];
  float4* slots = gather_slots();
  float acc[kIPT] = {0.f, 0.f, 0.f, 0.f}, dsum[kIPT] = {0.f, 0.f, 0.f, 0.f};
  LEnt<KIND> e[U];
  if constexpr (PIPE) {
#pragma unroll
    for (int u = 0; u < U; ++u) e[u] = l_load<KIND>(a, base + C * u + r, u < W, rr, q);
  }
  for (int32_t j = 0; j < W; j += U) {
    if constexpr (!PIPE) {
#pragma unroll
      for (int u = 0; u < U; ++u) e[u] = l_load<KIND>(a, base + C * (j + u) + r, j + u < W, rr, q);
    }
    float4 xv[SMEM ? 1 : U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if constexpr (SMEM) {
        if (j + u < W) gather_async(slots + u * kBBlock, X + (int64_t)e[u].c * TPR + q);
      } else {
        xv[u] = j + u < W ? X[(int64_t)e[u].c * TPR + q] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    LEnt<KIND> en[PIPE ? U : 1];
    if constexpr (PIPE) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        en[u] = l_load<KIND>(a, base + C * (j + U + u) + r, j + U + u < W, rr, q);
    }
    if constexpr (SMEM) gather_wait();
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j + u < W) {
        float4 x;
        if constexpr (SMEM) x = slots[u * kBBlock];
        else x = xv[u];
#pragma unroll
        for (int jj = 0; jj < kIPT; ++jj) {
          const float m = l_weight<KIND>(e[u], jj, st);
          if constexpr (KIND != kSets) dsum[jj] += m;
          acc[jj] = fmaf(m, get4(x, jj), acc[jj]);
        }
      }
    }
    if constexpr (PIPE) {
#pragma unroll
      for (int u = 0; u < U; ++u) e[u] = en[u];
    }
  }
  float4 y;
  if constexpr (KIND == kSets) {
    // CSR form: L_ii x_i + sum of (-w) x_c over free columns
    const float d = a.d32[rr];
#pragma unroll
    for (int jj = 0; jj < kIPT; ++jj) set4(y, jj, fmaf(d, get4(xi, jj), acc[jj]));
  } else {
    // edge form: sum of m (x_i - x_c); an identity row where all m are 0
#pragma unroll
    for (int jj = 0; jj < kIPT; ++jj)
      set4(y, jj, dsum[jj] == 0.0f ? get4(xi, jj) : fmaf(dsum[jj], get4(xi, jj), -acc[jj]));
  }
  return y;
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
struct GEnt {
  int32_t c;
  uint2 g;       // four BF16 values (per-instance factors) or one, repeated
};
__device__ __forceinline__ GEnt g_load(const BatchArgs& a, int h, int64_t p, bool ok,
                                       int32_t rr, int q) {
  GEnt e;
  e.c = ok ? __ldg(a.Gcol[h] + p) : rr;
  if (!ok) {
    e.g = make_uint2(0u, 0u);
  } else if (a.Gb[h]) {
    e.g = __ldg(reinterpret_cast<const uint2*>(a.Gb[h] + p * a.BS) + q);
  } else {
    const unsigned bits = __bfloat16_as_ushort(a.Gv[h][p]);
    e.g = make_uint2(bits | (bits << 16), bits | (bits << 16));
  }
  return e;
}

template <int U, bool SMEM, bool PIPE>
__device__ __forceinline__ float4 g_row(const BatchArgs& a, int h, int32_t base, int32_t W,
                                        int r, int q, int32_t row,
                                        const float4* __restrict__ X) {
  const int C = a.C, TPR = a.TPR;
  const int32_t rr = row >= 0 ? row : 0;
  float4* slots = gather_slots();
  float acc[kIPT] = {0.f, 0.f, 0.f, 0.f};
  GEnt e[U];
  if constexpr (PIPE) {
#pragma unroll
    for (int u = 0; u < U; ++u) e[u] = g_load(a, h, base + C * u + r, u < W, rr, q);
  }
  for (int32_t j = 0; j < W; j += U) {
    if constexpr (!PIPE) {
#pragma unroll
      for (int u = 0; u < U; ++u) e[u] = g_load(a, h, base + C * (j + u) + r, j + u < W, rr, q);
    }
    float4 xv[SMEM ? 1 : U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if constexpr (SMEM) {
        if (j + u < W) gather_async(slots + u * kBBlock, X + (int64_t)e[u].c * TPR + q);
      } else {
        xv[u] = j + u < W ? X[(int64_t)e[u].c * TPR + q] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    GEnt en[PIPE ? U : 1];
    if constexpr (PIPE) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        en[u] = g_load(a, h, base + C * (j + U + u) + r, j + U + u < W, rr, q);
    }
    if constexpr (SMEM) gather_wait();
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j + u < W) {
        float4 x;
        if constexpr (SMEM) x = slots[u * kBBlock];
        else x = xv[u];
        const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&e[u].g.x);
        const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&e[u].g.y);
        acc[0] = fmaf(__low2float(lo), x.x, acc[0]);
        acc[1] = fmaf(__high2float(lo), x.y, acc[1]);
        acc[2] = fmaf(__low2float(hi), x.z, acc[2]);
        acc[3] = fmaf(__high2float(hi), x.w, acc[3]);
      }
    }
    if constexpr (PIPE) {
#pragma unroll
      for (int u = 0; u < U; ++u) e[u] = en[u];
    }
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
// STAGE > 0: the FSAI halves (and, with STAGE_L, the SpMM) stream their
// structure through shared memory in chunks of STAGE entries, UG gathers
// per round trip; the other row products use U, SMEM and PIPE.
template <int KIND, int U, bool SMEM, bool PIPE, int STAGE = 0, bool STAGE_L = true,
          int UG = U>
__global__ void __launch_bounds__(kBBlock, 1)
pcg_batched_persistent(BatchArgs a) {
  static_assert(STAGE == 0 || (KIND == kSets && !SMEM), "staging: Dirichlet sets only");
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
  // whether a row-product phase runs for this lane: per lane (its quad has
  // an instance in `flags`), or, in the staged variants, whose warps copy
  // and synchronise together, for the whole warp (any lane's quad); the
  // extra lanes then compute products for instances that are not iterating,
  // which no later step reads (their step length is 0, their p is kept)
  auto phase_on = [&](const int* flags) {
    if constexpr (STAGE > 0) return __any_sync(0xffffffffu, any4(flags)) != 0;
    else return any4(flags) != 0;
  };
  // the slices of this block: one per warp in each window it owns.  Slices
  // are sorted by length inside a window, so the warp-to-slice assignment
  // rotates by 13 (coprime to 32) from window to window: every warp gets
  // long and short slices alike instead of warp 0 always the longest.
  auto windows = [&](const int32_t* perm, auto&& body) {
    int k = 0;
    for (int64_t win = blockIdx.x; win < a.nwin; win += gridDim.x, ++k) {
      const int64_t s = win * kBWarps + ((warp + 13 * k) & (kBWarps - 1));
      body(s, __ldg(perm + s * C + r));
    }
  };
  // The same, with lane 0 of each warp first prefetching into L2 what its
  // next slice (the block's next window) will read: the slice's structure
  // (pf_struct(s_next)) and a 1/32 share of the window's rows of the
  // vectors V0, V1 (gathered or read by row).  The prefetches run ahead on
  // the copy engine while the warp works on the current slice.
  const int64_t vq_win = (int64_t)kBWarps * C * TPR;             // float4 per window
  auto pf_rows = [&](const float4* V, int64_t nxt) {
    const int64_t share = vq_win / kBWarps;
    l2_prefetch(V + nxt * vq_win + warp * share, sizeof(float4) * share, V, V + n * TPR);
  };
  auto windows_pf = [&](const int32_t* perm, const int32_t* sptr, auto&& pf_struct,
                        const float4* V0, const float4* V1, auto&& body) {
    int64_t win = blockIdx.x;
    if (win >= a.nwin) return;
    int k = 0;
    auto slice_of = [&](int64_t w, int kk) {
      return w * kBWarps + ((warp + 13 * kk) & (kBWarps - 1));
    };
    int64_t s = slice_of(win, 0);
    int32_t row = __ldg(perm + s * C + r), b0 = __ldg(sptr + s), b1 = __ldg(sptr + s + 1);
    for (;;) {
      // the next window's slice indices are loaded now, so their latency
      // overlaps this window's work instead of starting the next one
      const int64_t nxt = win + gridDim.x;
      int64_t s2 = 0;
      int32_t row2 = -1, c0 = 0, c1 = 0;
      if (nxt < a.nwin) {
        s2 = slice_of(nxt, k + 1);
        row2 = __ldg(perm + s2 * C + r);
        c0 = __ldg(sptr + s2);
        c1 = __ldg(sptr + s2 + 1);
        if (lane == 0) {
          pf_struct(s2);
          if (V0) pf_rows(V0, nxt);
          if (V1) pf_rows(V1, nxt);
        }
      }
      body(b0, (b1 - b0) / C, row);
      if (nxt >= a.nwin) break;
      win = nxt;
      ++k;
      s = s2;
      row = row2;
      b0 = c0;
      b1 = c1;
    }
  };
  auto pf_L = [&](int64_t sn) {
    const int64_t b0 = a.Lsptr[sn], b1 = a.Lsptr[sn + 1];
    if constexpr (KIND == kFields) {
      l2_prefetch(a.Lcol + b0, 4 * (b1 - b0), a.Lcol, a.Lcol + a.Ltotal);
      l2_prefetch(a.Lw + b0 * BS, 4 * BS * (b1 - b0), a.Lw, a.Lw + a.Ltotal * BS);
    } else {
      l2_prefetch(a.Lcw + b0, 8 * (b1 - b0), a.Lcw, a.Lcw + a.Ltotal);
      if constexpr (KIND == kStates) l2_prefetch(a.Lfc + b0, b1 - b0, a.Lfc, a.Lfc + a.Ltotal);
    }
  };
  auto pf_G = [&](int h, int64_t sn) {
    const int64_t b0 = a.Gsptr[h][sn], b1 = a.Gsptr[h][sn + 1];
    l2_prefetch(a.Gcol[h] + b0, 4 * (b1 - b0), a.Gcol[h], a.Gcol[h] + a.Gtotal[h]);
    if (a.Gb[h])
      l2_prefetch(a.Gb[h] + b0 * BS, 2 * BS * (b1 - b0), a.Gb[h], a.Gb[h] + a.Gtotal[h] * BS);
    else
      l2_prefetch(a.Gv[h] + b0, 2 * (b1 - b0), a.Gv[h], a.Gv[h] + a.Gtotal[h]);
  };
  // Staged streaming (STAGE = K entries per chunk): the windows and
  // prefetches of windows_pf; the structure arrays A0 (eb0 bytes per entry)
  // and A1 (eb1, or none) of each slice go through the warp's double buffer.
  // consume(chunk, nent, acc) adds nent entries of the chunk (A0's part at
  // offset 0, A1's at K * C * eb0) to the row's accumulators; finish(row,
  // acc) completes a row.  Every lane of a warp takes the same path.
  auto staged = [&](const int32_t* perm, const int32_t* sptr, auto&& pf_struct,
                    const float4* V0, const float4* V1, const char* A0, int eb0,
                    const char* A1, int eb1, auto&& consume, auto&& finish) {
    int64_t win = blockIdx.x;
    if (win >= a.nwin) return;
    extern __shared__ __align__(16) float4 bsm_slots[];
    const int chunk = STAGE * C * (STAGE_L ? 8 : 6);
    char* wb = reinterpret_cast<char*>(bsm_slots) + (size_t)warp * 2 * chunk;
    auto copy_chunk = [&](int32_t b0, int j0, int nent, int buf) {
      char* d = wb + buf * chunk;
      const char* s0 = A0 + ((int64_t)b0 + (int64_t)C * j0) * eb0;
      const int n0 = nent * C * eb0 / 16;
      for (int i = lane; i < n0; i += 32) copy16_async(d + 16 * i, s0 + 16 * i);
      if (A1) {
        const char* s1 = A1 + ((int64_t)b0 + (int64_t)C * j0) * eb1;
        char* d1 = d + STAGE * C * eb0;
        const int n1 = nent * C * eb1 / 16;
        for (int i = lane; i < n1; i += 32) copy16_async(d1 + 16 * i, s1 + 16 * i);
      }
    };
    int k = 0;
    auto slice_of = [&](int64_t w, int kk) {
      return w * kBWarps + ((warp + 13 * kk) & (kBWarps - 1));
    };
    int64_t s = slice_of(win, 0);
    int32_t row = __ldg(perm + s * C + r), b0 = __ldg(sptr + s);
    int32_t W = (__ldg(sptr + s + 1) - b0) / C;
    int cb = 0;
    bool have = false;          // this slice's first chunk is already in buffer cb
    for (;;) {
      const int64_t nxt = win + gridDim.x;
      int32_t row2 = -1, c0 = 0, W2 = 0;
      if (nxt < a.nwin) {
        const int64_t s2 = slice_of(nxt, k + 1);
        row2 = __ldg(perm + s2 * C + r);
        c0 = __ldg(sptr + s2);
        W2 = (__ldg(sptr + s2 + 1) - c0) / C;
        if (lane == 0) {
          pf_struct(s2);
          if (V0) pf_rows(V0, nxt);
          if (V1) pf_rows(V1, nxt);
        }
      }
      float acc[kIPT] = {0.f, 0.f, 0.f, 0.f};
      bool next_have = false;
      if (W > 0) {
        if (!have) {
          copy_chunk(b0, 0, min(STAGE, W), cb);
          copy_commit();
        }
        for (int j0 = 0; j0 < W; j0 += STAGE) {
          const int nent = min(STAGE, W - j0);
          next_have = false;
          if (j0 + STAGE < W) {
            copy_chunk(b0, j0 + STAGE, min(STAGE, W - j0 - STAGE), cb ^ 1);
          } else if (W2 > 0) {
            copy_chunk(c0, 0, min(STAGE, W2), cb ^ 1);
            next_have = true;
          }
          copy_commit();
          copy_wait<1>();
          __syncwarp();
          consume(wb + cb * chunk, nent, acc);
          __syncwarp();
          cb ^= 1;
        }
      }
      have = next_have;
      finish(row, acc);
      if (nxt >= a.nwin) break;
      win = nxt;
      ++k;
      row = row2;
      b0 = c0;
      W = W2;
    }
    copy_wait<0>();
    __syncwarp();
  };
  // chunk consumers of the staged variants: L of Dirichlet sets ((column,
  // FP32 value) pairs) and an FSAI half (columns, then BF16 values), in
  // entry order with the FMAs of l_row / g_row, so results are bit-identical
  auto consume_L = [=](const float4* __restrict__ Xv, const char* ch, int nent,
                       float (&acc)[kIPT]) {
    const int2* e = reinterpret_cast<const int2*>(ch);
    for (int u0 = 0; u0 < nent; u0 += UG) {
      float4 xv[UG];
      float wv[UG];
#pragma unroll
      for (int u = 0; u < UG; ++u) {
        wv[u] = 0.0f;
        xv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (u0 + u < nent) {
          const int2 cw = e[(u0 + u) * C + r];
          wv[u] = __int_as_float(cw.y);
          xv[u] = Xv[(int64_t)cw.x * TPR + q];
        }
      }
#pragma unroll
      for (int u = 0; u < UG; ++u) {
        if (u0 + u < nent) {
          acc[0] = fmaf(wv[u], xv[u].x, acc[0]);
          acc[1] = fmaf(wv[u], xv[u].y, acc[1]);
          acc[2] = fmaf(wv[u], xv[u].z, acc[2]);
          acc[3] = fmaf(wv[u], xv[u].w, acc[3]);
        }
      }
    }
  };
  auto consume_G = [=](const float4* __restrict__ Xv, const char* ch, int nent,
                       float (&acc)[kIPT]) {
    const int32_t* col = reinterpret_cast<const int32_t*>(ch);
    const __nv_bfloat16* gv = reinterpret_cast<const __nv_bfloat16*>(ch + STAGE * C * 4);
    for (int u0 = 0; u0 < nent; u0 += UG) {
      float4 xv[UG];
      float gw[UG];
#pragma unroll
      for (int u = 0; u < UG; ++u) {
        gw[u] = 0.0f;
        xv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (u0 + u < nent) {
          gw[u] = __bfloat162float(gv[(u0 + u) * C + r]);
          xv[u] = Xv[(int64_t)col[(u0 + u) * C + r] * TPR + q];
        }
      }
#pragma unroll
      for (int u = 0; u < UG; ++u) {
        if (u0 + u < nent) {
          acc[0] = fmaf(gw[u], xv[u].x, acc[0]);
          acc[1] = fmaf(gw[u], xv[u].y, acc[1]);
          acc[2] = fmaf(gw[u], xv[u].z, acc[2]);
          acc[3] = fmaf(gw[u], xv[u].w, acc[3]);
        }
      }
    }
  };
  // device time of the phases of the FP32 iterations, taken by thread 0 of
  // block 0 as it leaves each grid barrier (every block leaves a barrier at
  // about the same time): SpMM, x/r update, FSAI lower half, upper half,
  // p update
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  __shared__ unsigned long long t_last;
  __shared__ double ph[6];                 // [5]: iterations timed
  if (timer) {
    t_last = 0;
    for (int k = 0; k < 6; ++k) ph[k] = 0.0;
  }
  auto mark = [&](int k) {
    if (!timer) return;
    const unsigned long long t = global_ns();
    if (k >= 0) ph[k] += (double)(t - t_last);
    t_last = t;
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
  auto apply_precond = [&](const int* flags, bool timed) -> bool {
    if (phase_on(flags)) {
      if constexpr (STAGE > 0) {
        staged(a.Gperm[0], a.Gsptr[0], [&](int64_t sn) { pf_G(0, sn); }, R, nullptr,
               reinterpret_cast<const char*>(a.Gcol[0]), 4,
               reinterpret_cast<const char*>(a.Gv[0]), 2,
               [&](const char* ch, int nent, float (&y)[kIPT]) { consume_G(R, ch, nent, y); },
               [&](int32_t row, float (&y)[kIPT]) {
          if (row >= 0) T[(int64_t)row * TPR + q] = make_float4(y[0], y[1], y[2], y[3]);
        });
      } else {
        windows_pf(a.Gperm[0], a.Gsptr[0], [&](int64_t sn) { pf_G(0, sn); }, R, nullptr,
                   [&](int32_t base, int32_t W, int32_t row) {
          const float4 y = g_row<U, SMEM, PIPE>(a, 0, base, W, r, q, row, R);
          if (row >= 0) T[(int64_t)row * TPR + q] = y;
        });
      }
    }
    if (!bgrid_sync(a.bar, err)) return false;
    if (timed) mark(2);
    Acc2 acc[kIPT];
    if (phase_on(flags)) {
      auto upper_row = [&](int32_t row, const float4 zi) {
        if (row < 0) return;
        Z[(int64_t)row * TPR + q] = zi;
        const float4 ri = R[(int64_t)row * TPR + q];
#pragma unroll
        for (int j = 0; j < kIPT; ++j) acc[j].add(get4(ri, j), get4(zi, j));
      };
      if constexpr (STAGE > 0) {
        staged(a.Gperm[1], a.Gsptr[1], [&](int64_t sn) { pf_G(1, sn); }, T, R,
               reinterpret_cast<const char*>(a.Gcol[1]), 4,
               reinterpret_cast<const char*>(a.Gv[1]), 2,
               [&](const char* ch, int nent, float (&y)[kIPT]) { consume_G(T, ch, nent, y); },
               [&](int32_t row, float (&y)[kIPT]) {
          upper_row(row, make_float4(y[0], y[1], y[2], y[3]));
        });
      } else {
        windows_pf(a.Gperm[1], a.Gsptr[1], [&](int64_t sn) { pf_G(1, sn); }, T, R,
                   [&](int32_t base, int32_t W, int32_t row) {
          upper_row(row, g_row<U, SMEM, PIPE>(a, 1, base, W, r, q, row, T));
        });
      }
    }
    double v[kIPT];
#pragma unroll
    for (int j = 0; j < kIPT; ++j) v[j] = acc[j].get();
    if (!breduce(v, a, parity, S, shw, err)) return false;
    if (timed) mark(3);
    return true;
  };

  for (;;) {
    // ---- segment start for the active instances: z = M r, p = z + beta p
    if (!apply_precond(S.active, false)) return;
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
    mark(-1);

    // ---- FP32 iterations until every working instance is frozen
    for (;;) {
      {
        Acc2 acc[kIPT];
        if (phase_on(S.iterating)) {
          auto spmm_row = [&](int32_t row, const float4 qi) {
            if (row < 0) return;
            Q[(int64_t)row * TPR + q] = qi;
            const float4 pi = Pv[(int64_t)row * TPR + q];
#pragma unroll
            for (int j = 0; j < kIPT; ++j) acc[j].add(get4(pi, j), get4(qi, j));
          };
          if constexpr (STAGE > 0 && STAGE_L) {
            // CSR form of the Dirichlet sets: L_ii x_i + the staged entries
            staged(a.Lperm, a.Lsptr, pf_L, Pv, nullptr, reinterpret_cast<const char*>(a.Lcw),
                   8, nullptr, 0,
                   [&](const char* ch, int nent, float (&y)[kIPT]) { consume_L(Pv, ch, nent, y); },
                   [&](int32_t row, float (&y)[kIPT]) {
              const int32_t rr = row >= 0 ? row : 0;
              const float4 xi = Pv[(int64_t)rr * TPR + q];
              const float d = a.d32[rr];
              spmm_row(row, make_float4(fmaf(d, xi.x, y[0]), fmaf(d, xi.y, y[1]),
                                        fmaf(d, xi.z, y[2]), fmaf(d, xi.w, y[3])));
            });
          } else {
            windows_pf(a.Lperm, a.Lsptr, pf_L, Pv, nullptr,
                       [&](int32_t base, int32_t W, int32_t row) {
              spmm_row(row, l_row<KIND, U, SMEM, PIPE>(a, base, W, r, q, row, st, Pv));
            });
          }
        }
        double v[kIPT];
#pragma unroll
        for (int j = 0; j < kIPT; ++j) v[j] = acc[j].get();
        if (!breduce(v, a, parity, S, shw, err)) return;
        mark(0);
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
        mark(1);
      }
      if (threadIdx.x < BS) {
        const int i = threadIdx.x;
        if (S.iterating[i]) {
          S.iters[i] += 1;
          const double rr = S.red[i];
          if (rr <= S.tol2[i] || S.iters[i] >= a.max_iter || !isfinite(rr)) S.iterating[i] = 0;
        }
      }
      __syncthreads();   // instances 32..63 are updated by warp 1: count after both
      if (threadIdx.x == 0) {
        int c = 0;
        for (int i = 0; i < BS; ++i) c += S.iterating[i];
        S.count = c;
      }
      __syncthreads();
      if (S.count == 0) break;
      // preconditioner on the iterating instances
      if (!apply_precond(S.iterating, true)) return;
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
      mark(4);
      if (timer) ph[5] += 1.0;
    }
    mark(-1);

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
    __syncthreads();   // as above: every instance updated before the count
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
  if (timer) {
    for (int k = 0; k < 5; ++k) a.phase[k] = ph[k] * 1e-6;   // ms
    a.phase[5] = ph[5];
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

// Sort key of a node for the batched numbering: the box is cut into
// 2^t x 2^t x 2^t tiles, taken in natural order (x fastest, then y, z), and
// the nodes of a tile in Morton order of their position inside it (21 - t
// bits per coordinate, interleaved, x lowest).  Inside a tile the order is
// compact, so a window of consecutive nodes is a small patch; across tiles
// it sweeps the box in slabs, so the patches worked on at the same time, and
// their neighbours, are close together.
__global__ void morton_keys_kernel(int64_t n, const double* __restrict__ xyz, double3 lo,
                                   double3 scale, int t, uint64_t* __restrict__ key,
                                   uint32_t* __restrict__ val) {
  const int lb = 21 - t;                                 // bits inside a tile
  const uint64_t lmask = (1ull << lb) - 1ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double fx = (xyz[3 * i] - lo.x) * scale.x;
    const double fy = (xyz[3 * i + 1] - lo.y) * scale.y;
    const double fz = (xyz[3 * i + 2] - lo.z) * scale.z;
    const uint64_t ix = (uint64_t)fmin(fmax(fx, 0.0), 2097151.0);
    const uint64_t iy = (uint64_t)fmin(fmax(fy, 0.0), 2097151.0);
    const uint64_t iz = (uint64_t)fmin(fmax(fz, 0.0), 2097151.0);
    const uint64_t tile = (((iz >> lb) << (2 * t)) | ((iy >> lb) << t) | (ix >> lb));
    const uint64_t in = spread21(ix & lmask) | (spread21(iy & lmask) << 1) |
                        (spread21(iz & lmask) << 2);
    key[i] = (tile << (3 * lb)) | in;
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

// bounding box of the nodes: per-block (min x, min y, min z, max x, max y,
// max z) into part[6 * block], then one block folds the partials into out
__global__ void bbox_kernel(int64_t n, const double* __restrict__ xyz, double* __restrict__ part) {
  __shared__ double sh[6][256];
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int d = 0; d < 3; ++d) {
      lo[d] = fmin(lo[d], xyz[3 * i + d]);
      hi[d] = fmax(hi[d], xyz[3 * i + d]);
    }
  for (int d = 0; d < 3; ++d) {
    sh[d][threadIdx.x] = lo[d];
    sh[3 + d][threadIdx.x] = hi[d];
  }
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int d = 0; d < 3; ++d) {
        sh[d][threadIdx.x] = fmin(sh[d][threadIdx.x], sh[d][threadIdx.x + h]);
        sh[3 + d][threadIdx.x] = fmax(sh[3 + d][threadIdx.x], sh[3 + d][threadIdx.x + h]);
      }
    __syncthreads();
  }
  if (threadIdx.x < 6) part[6 * (int64_t)blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void bbox_fold_kernel(int nb, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x < 6) {
    double v = part[threadIdx.x];
    for (int b = 1; b < nb; ++b)
      v = threadIdx.x < 3 ? fmin(v, part[6 * b + threadIdx.x]) : fmax(v, part[6 * b + threadIdx.x]);
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

// Node order of the batched layouts: Morton order inside tiles of about
// kTileNodes nodes, tiles in natural order
#ifndef DEC_TILE_NODES
#define DEC_TILE_NODES 1024
#endif
constexpr int kTileNodes = DEC_TILE_NODES;
static dec_status build_morton(dec_ctx* ctx) {
  const int64_t n = ctx->n;
  cudaStream_t s = ctx->stream;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, ctx->num_sms * 4));
  DEC_TRY(ctx->kpartial.ensure(6 * (size_t)nb + 8));
  bbox_kernel<<<nb, 256, 0, s>>>(n, ctx->xyz.p, ctx->kpartial.p + 8);
  bbox_fold_kernel<<<1, 32, 0, s>>>(nb, ctx->kpartial.p + 8, ctx->kpartial.p);
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
  // tiles of about kTileNodes nodes: 2^t per axis, t = floor(log2(cbrt(n / kTileNodes)))
  int t = 0;
  while (t < 10 && (double)(1 << (3 * (t + 1))) * kTileNodes <= (double)n) ++t;
  morton_keys_kernel<<<grid_for_work(ctx, n), 256, 0, s>>>(n, ctx->xyz.p, lo, sc, t,
                                                           ctx->key_a.p, ctx->val_a.p);
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

// Kernel variants for the context's instance kind: entries per round trip
// (U), whether the next round's structure loads overlap the gathers, where
// the gathers go (registers or shared memory), and for Dirichlet sets the
// staged variants (structure through shared memory, K entries per chunk);
// reported as 1000 * K / 8 + 100 * shared + 10 * overlapped + U, plus 500
// when only the FSAI halves are staged (the SpMM then runs as the variant
// 10 * overlapped + U, the staged halves with 4 gathers per round trip).
// All variants of a kind add a row's entries in the same order, so the
// choice never changes a result.
constexpr int kNumGatherVariants = 9;
constexpr int kGatherVariants[kNumGatherVariants] = {2,    4,    12,   114, 106,
                                                     1004, 2004, 2002, 2512};
constexpr int kStageEntries[kNumGatherVariants] = {0, 0, 0, 0, 0, 8, 16, 16, 16};

bool batch_variant_code(int code) {
  for (int c = 0; c < kNumGatherVariants; ++c)
    if (kGatherVariants[c] == code) return true;
  return false;
}

static int variant_smem(int v, int C) {
  switch (v) {
    case 3: return gather_smem<4>();
    case 4: return gather_smem<6>();
    case 5: return stage_smem<8>(C);
    case 6:
    case 7: return stage_smem<16>(C);
    case 8: return stage_smem<16>(C, 6);   // FSAI entries only
    default: return 0;
  }
}

template <int KIND>
static const void* batch_kernel(int v) {
  switch (v) {
    case 0: return (const void*)pcg_batched_persistent<KIND, 2, false, false>;
    case 1: return (const void*)pcg_batched_persistent<KIND, 4, false, false>;
    case 2: return (const void*)pcg_batched_persistent<KIND, 2, false, true>;
    case 3: return (const void*)pcg_batched_persistent<KIND, 4, true, true>;
    case 4: return (const void*)pcg_batched_persistent<KIND, 6, true, false>;
    default: break;
  }
  if constexpr (KIND == kSets) {
    switch (v) {
      case 5: return (const void*)pcg_batched_persistent<KIND, 4, false, false, 8>;
      case 6: return (const void*)pcg_batched_persistent<KIND, 4, false, false, 16>;
      case 7: return (const void*)pcg_batched_persistent<KIND, 2, false, false, 16>;
      case 8: return (const void*)pcg_batched_persistent<KIND, 2, false, true, 16, false, 4>;
      default: break;
    }
  }
  return nullptr;
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
  int smem[kNumGatherVariants];
  bool any = false;
  const int Cb = 32 / (BS / kIPT);
  for (int v = 0; v < kNumGatherVariants; ++v) {
    smem[v] = variant_smem(v, Cb);
    usable[v] = false;
    // staged copies move 16 bytes: C rows of a BF16 value must fill them
    if (!kern[v] || (kStageEntries[v] > 0 && Cb < 8)) continue;
    int per_sm = 0;
    DEC_TRY(cudaFuncSetAttribute(kern[v], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem[v]));
    DEC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern[v], kBBlock, smem[v]));
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
  double* phase = reinterpret_cast<double*>(ctx->coop.p + 16 + kBMax / 2 + 2 * kBMax);
  BatchArgs a{};
  a.phase = phase;
  a.n = n;
  a.B = B;
  a.BS = BS;
  a.TPR = BS / kIPT;
  a.C = 32 / a.TPR;
  a.nwin = (n + ctx->bL.R - 1) / ctx->bL.R;
  a.Ltotal = ctx->bL.total;
  a.Gtotal[0] = ctx->bGlo.total;
  a.Gtotal[1] = ctx->bGup.total;
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
      e = cudaLaunchCooperativeKernel(kern[v], dim3(grid), dim3(kBBlock), args, smem[v], s);
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
  if (ctx->batch_force != 0) {
    // a variant chosen by the caller (dec_set_batch_variant): no tuning
    v = -1;
    for (int c = 0; c < kNumGatherVariants; ++c)
      if (kGatherVariants[c] == ctx->batch_force && usable[c]) v = c;
    if (v < 0)
      return ctx->fail(DEC_ERR_ARG, "batched solve: the chosen variant does not fit this batch");
  }
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
      e = cudaLaunchCooperativeKernel(kern[v], dim3(grid), dim3(kBBlock), args, smem[v], s);
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
  DEC_TRY(cudaMemcpyAsync(ctx->batch_phase_ms, phase, sizeof(double) * 6,
                          cudaMemcpyDeviceToHost, s));
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
