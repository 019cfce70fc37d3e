// dec_batch.cu - many instances on one mesh in one persistent launch: the
// crack states of a growing disc population (each state zeroes the *1 of the
// edges it cuts, Sec. 2.5) or several Dirichlet value sets, solved together
// by mixed-precision PCG over a sparse matrix - multiple vector product.
//
// The instances share L's sparsity; vectors are stored node-major with the
// instances contiguous (X[i * BS + b], BS = padded instance count), so one
// gathered neighbour row X[c][0..BS) is one coalesced load.  Each thread
// handles four consecutive instances of a row (16-byte loads), so BS / 4
// threads share a row and the per-entry structure is read once per four
// instances.  The operator of instance b is applied in "edge form" from
// shared per-entry data (column, *1 in FP32 and FP64, first crack state):
//   (L_b x)_i = sum_k w_k [b < fc_k] (x_i - x_c),
// which needs no per-instance values or diagonal (vectors are zero on
// Dirichlet nodes, so those columns drop out; Dirichlet rows and rows whose
// weights are all zero in instance b are identity rows).  Dirichlet value
// sets share the FSAI factor of L; crack states each get their own factor,
// computed in FP32 and stored in BF16 with the instances contiguous.
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

namespace dec {

constexpr int kBBlock = 1024;             // one block of 1024 threads per SM
constexpr int kBMax = 64;                 // instances per batched launch
constexpr long kBSpinLimit = 1L << 24;

struct BatchArgs {
  int64_t n;
  int B, BS;                              // instances, padded stride (8..64)
  const int32_t* rowptr;
  const int32_t* col;
  const int32_t* dpos;
  const uint8_t* tag;
  const float* w32;                       // [nnz] *1 of the entry's edge (0 on the diagonal)
  const double* w64;
  const uint8_t* fc;                      // [nnz] first crack state (255: never)
  int states;                             // 1: instance b is crack state b; 0: all state 0
  const __nv_bfloat16* g;                 // [nnz] shared FSAI factor, CSR layout
  const __nv_bfloat16* gb;                // [nnz][BS] per-instance factors, or nullptr
  const double* bvec;                     // [n][BS]
  double *x64, *r64;                      // [n][BS]
  float *x, *r, *z, *p, *q, *t;           // [n][BS]
  double* partial;                        // [2][2][grid][BS]
  unsigned* bar;
  int* status;                            // [0] error
  int* iters;                             // [BS]
  double* result;                         // [BS] final rr, [BS] |b|^2
  double rtol2, seg2;
  int max_iter;
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
  double red[2][kBMax];          // results of the last reduction
  float alpha[kBMax], beta[kBMax];
  int active[kBMax];             // still solving
  int iterating[kBMax];          // active and not frozen in this segment
  int restart[kBMax];
  int stall[kBMax];
  int iters[kBMax];
  int count;                     // scratch: number of iterating instances
};

// Each thread works on four instances (one float4 of a node's row of a
// batched vector): a row of BS instances is handled by TPR = BS / 4 threads.
// The per-entry structure (column, weight, crack state) is loaded once per
// four instances and the gathers are 16-byte loads.
constexpr int kIPT = 4;

// Per-instance grid reduction of NV quantities; thread t contributes v[k][j]
// to instance 4 (t % TPR) + j.  Results land in S.red[k][b], identical in
// every block.
template <int NV>
__device__ bool breduce(const double (&v)[NV][kIPT], double* partial, int& parity, BState& S,
                        double* sh, int BS, unsigned* bar, int* err) {
  const int G = gridDim.x;
  const int TPR = BS / kIPT;
  double* part = partial + (size_t)parity * 2 * G * BS;
  parity ^= 1;
  const int rows = kBBlock / TPR;                 // threads sharing an instance quad
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int j = 0; j < kIPT; ++j) sh[threadIdx.x * kIPT + j] = v[k][j];
    __syncthreads();
    if (threadIdx.x < BS) {
      const int q = threadIdx.x / kIPT, j = threadIdx.x % kIPT;
      double s = 0.0;
      for (int m = 0; m < rows; ++m) s += sh[(q + m * TPR) * kIPT + j];
      part[((size_t)k * G + blockIdx.x) * BS + threadIdx.x] = s;
    }
    __syncthreads();
  }
  if (!bgrid_sync(bar, err)) return false;
  const int per = kBBlock / BS;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const int b = threadIdx.x % BS, slot = threadIdx.x / BS;
    double s = 0.0;
    for (int blk = slot; blk < G; blk += per)
      s += __ldcg(part + ((size_t)k * G + blk) * BS + b);
    sh[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < BS) {
      double tot = 0.0;
      for (int j = 0; j < per; ++j) tot += sh[threadIdx.x + j * BS];
      S.red[k][threadIdx.x] = tot;
    }
    __syncthreads();
  }
  return true;
}

__device__ __forceinline__ float get4(const float4& v, int j) {
  return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}
__device__ __forceinline__ void set4(float4& v, int j, float x) {
  if (j == 0) v.x = x; else if (j == 1) v.y = x; else if (j == 2) v.z = x; else v.w = x;
}

// The gathers of the FP32 row products can go to shared memory with
// 16-byte asynchronous copies: registers (64 per thread at 1024 threads per
// SM) then do not bound the gathers in flight, and a row takes
// ceil(entries / kGU) round trips instead of ceil(entries / 4).  Slot u of
// thread t is slots[u * 1024 + t] (conflict-free 16-byte accesses); a thread
// reads only its own slots, so no barrier is needed.  The shared memory
// comes out of L1, which costs more than it gains when few threads share a
// row (8 instances); the autotuner in solve_batched picks the variant.
// Gather variants of the batched kernel (the autotuner picks one per
// problem, see solve_batched): 0 = register gathers, 4 at a time; G > 0 =
// shared-memory gathers, G entries per round trip.
constexpr int kGatherVariants[] = {0, 4, 6, 8};
constexpr int kNumGatherVariants = 4;
template <int GU>
constexpr int gather_smem() { return GU * kBBlock * (int)sizeof(float4); }

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

// (L_b x)_i for the four instances 4q..4q+3 of row i (FP32).  The diagonal
// slot carries w = 0, so it needs no test.
template <int kGU>
__device__ __forceinline__ float4 edge_form4_async(const BatchArgs& a, int64_t i, int q,
                                             const int (&st)[kIPT],
                                             const float4* __restrict__ X) {
  const int TPR = a.BS / kIPT;
  float4* slots = gather_slots();
  const float4 xi = X[i * TPR + q];
  if (a.tag[i] == DEC_NODE_DIRICHLET) return xi;
  const int32_t k0 = a.rowptr[i], k1 = a.rowptr[i + 1];
  float acc[kIPT] = {0.f, 0.f, 0.f, 0.f}, dsum[kIPT] = {0.f, 0.f, 0.f, 0.f};
  for (int32_t k = k0; k < k1; k += kGU) {
    const int cnt = k1 - k < kGU ? k1 - k : kGU;
    int32_t c[kGU];
#pragma unroll
    for (int u = 0; u < kGU; ++u) c[u] = u < cnt ? __ldg(a.col + k + u) : 0;
#pragma unroll
    for (int u = 0; u < kGU; ++u)
      if (u < cnt) gather_async(slots + u * kBBlock, X + (int64_t)c[u] * TPR + q);
    float wv[kGU];
    int f[kGU];
#pragma unroll
    for (int u = 0; u < kGU; ++u) {
      wv[u] = u < cnt ? __ldg(a.w32 + k + u) : 0.0f;
      f[u] = u < cnt ? (int)__ldg(a.fc + k + u) : 0;
    }
    gather_wait();
#pragma unroll
    for (int u = 0; u < kGU; ++u) {
      if (u < cnt) {
        const float4 xv = slots[u * kBBlock];
#pragma unroll
        for (int j = 0; j < kIPT; ++j) {
          const float m = f[u] > st[j] ? wv[u] : 0.0f;
          dsum[j] += m;
          acc[j] = fmaf(m, get4(xv, j), acc[j]);
        }
      }
    }
  }
  float4 y;
#pragma unroll
  for (int j = 0; j < kIPT; ++j)
    set4(y, j, dsum[j] == 0.0f ? get4(xi, j) : fmaf(dsum[j], get4(xi, j), -acc[j]));
  return y;
}

// (L_b x)_i for the four instances 4q..4q+3 of row i (FP32), gathers into
// registers 4 at a time (the path for small instance strides).  Entries are
// taken 4 at a time: structure loads, then 4 independent 16-byte gathers.
// The diagonal slot carries w = 0, so it needs no test.
__device__ __forceinline__ float4 edge_form4_reg(const BatchArgs& a, int64_t i, int q,
                                             const int (&st)[kIPT],
                                             const float4* __restrict__ X) {
  constexpr int U = 4;
  const int TPR = a.BS / kIPT;
  const float4 xi = X[i * TPR + q];
  if (a.tag[i] == DEC_NODE_DIRICHLET) return xi;
  const int32_t k0 = a.rowptr[i], k1 = a.rowptr[i + 1];
  float acc[kIPT] = {0.f, 0.f, 0.f, 0.f}, dsum[kIPT] = {0.f, 0.f, 0.f, 0.f};
  for (int32_t k = k0; k < k1; k += U) {
    int32_t c[U];
    float wv[U];
    int f[U];
    float4 xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = k + u < k1;
      c[u] = ok ? __ldg(a.col + k + u) : 0;
      wv[u] = ok ? __ldg(a.w32 + k + u) : 0.0f;
      f[u] = ok ? (int)__ldg(a.fc + k + u) : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      xv[u] = k + u < k1 ? X[(int64_t)c[u] * TPR + q] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < kIPT; ++j) {
        const float m = f[u] > st[j] ? wv[u] : 0.0f;
        dsum[j] += m;
        acc[j] = fmaf(m, get4(xv[u], j), acc[j]);
      }
  }
  float4 y;
#pragma unroll
  for (int j = 0; j < kIPT; ++j)
    set4(y, j, dsum[j] == 0.0f ? get4(xi, j) : fmaf(dsum[j], get4(xi, j), -acc[j]));
  return y;
}

// The same in FP64 (the residual of a reliable update), x64 as double
__device__ __forceinline__ void edge_form4_64(const BatchArgs& a, int64_t i, int q,
                                              const int (&st)[kIPT],
                                              const double* __restrict__ X, double (&y)[kIPT]) {
  const int BS = a.BS;
  const double* xi = X + i * BS + kIPT * q;
  if (a.tag[i] == DEC_NODE_DIRICHLET) {
#pragma unroll
    for (int j = 0; j < kIPT; ++j) y[j] = xi[j];
    return;
  }
  double acc[kIPT] = {0.0, 0.0, 0.0, 0.0}, dsum[kIPT] = {0.0, 0.0, 0.0, 0.0};
  for (int32_t k = a.rowptr[i]; k < a.rowptr[i + 1]; ++k) {
    const int32_t c = __ldg(a.col + k);
    const double wk = __ldg(a.w64 + k);
    const int f = (int)__ldg(a.fc + k);
    const double2 x01 = *reinterpret_cast<const double2*>(X + (int64_t)c * BS + kIPT * q);
    const double2 x23 = *reinterpret_cast<const double2*>(X + (int64_t)c * BS + kIPT * q + 2);
    const double xc[kIPT] = {x01.x, x01.y, x23.x, x23.y};
#pragma unroll
    for (int j = 0; j < kIPT; ++j) {
      const double m = f > st[j] ? wk : 0.0;
      dsum[j] += m;
      acc[j] = fma(m, xc[j], acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < kIPT; ++j) y[j] = dsum[j] == 0.0 ? xi[j] : fma(dsum[j], xi[j], -acc[j]);
}

// FSAI halves (lower: G, upper: G^T) for four instances; per-instance
// factors (gb) or the shared one (g); gathers as in edge_form4
template <int kGU>
__device__ __forceinline__ float4 fsai4_async(const BatchArgs& a, int64_t i, int q, bool lower,
                                        const float4* __restrict__ X) {
  const int BS = a.BS, TPR = BS / kIPT;
  float4* slots = gather_slots();
  const int32_t k0 = lower ? a.rowptr[i] : a.dpos[i];
  const int32_t k1 = lower ? a.dpos[i] + 1 : a.rowptr[i + 1];
  float acc[kIPT] = {0.f, 0.f, 0.f, 0.f};
  for (int32_t k = k0; k < k1; k += kGU) {
    const int cnt = k1 - k < kGU ? k1 - k : kGU;
    int32_t c[kGU];
#pragma unroll
    for (int u = 0; u < kGU; ++u) c[u] = u < cnt ? __ldg(a.col + k + u) : 0;
#pragma unroll
    for (int u = 0; u < kGU; ++u)
      if (u < cnt) gather_async(slots + u * kBBlock, X + (int64_t)c[u] * TPR + q);
    uint2 graw[kGU];
#pragma unroll
    for (int u = 0; u < kGU; ++u) {
      if (u >= cnt) {
        graw[u] = make_uint2(0u, 0u);
      } else if (a.gb) {
        graw[u] = *reinterpret_cast<const uint2*>(a.gb + (int64_t)(k + u) * BS + kIPT * q);
      } else {
        const unsigned bits = __bfloat16_as_ushort(a.g[k + u]);
        graw[u] = make_uint2(bits | (bits << 16), bits | (bits << 16));
      }
    }
    gather_wait();
#pragma unroll
    for (int u = 0; u < kGU; ++u) {
      if (u < cnt) {
        const float4 xv = slots[u * kBBlock];
        const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&graw[u].x);
        const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&graw[u].y);
        acc[0] = fmaf(__low2float(lo), xv.x, acc[0]);
        acc[1] = fmaf(__high2float(lo), xv.y, acc[1]);
        acc[2] = fmaf(__low2float(hi), xv.z, acc[2]);
        acc[3] = fmaf(__high2float(hi), xv.w, acc[3]);
      }
    }
  }
  return make_float4(acc[0], acc[1], acc[2], acc[3]);
}

// FSAI halves with register gathers (small instance strides)
__device__ __forceinline__ float4 fsai4_reg(const BatchArgs& a, int64_t i, int q, bool lower,
                                        const float4* __restrict__ X) {
  constexpr int U = 4;
  const int BS = a.BS, TPR = BS / kIPT;
  const int32_t k0 = lower ? a.rowptr[i] : a.dpos[i];
  const int32_t k1 = lower ? a.dpos[i] + 1 : a.rowptr[i + 1];
  float acc[kIPT] = {0.f, 0.f, 0.f, 0.f};
  for (int32_t k = k0; k < k1; k += U) {
    int32_t c[U];
    float g[U][kIPT];
    float4 xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = k + u < k1;
      c[u] = ok ? __ldg(a.col + k + u) : 0;
      if (!ok) {
#pragma unroll
        for (int j = 0; j < kIPT; ++j) g[u][j] = 0.0f;
      } else if (a.gb) {
        const uint2 raw = *reinterpret_cast<const uint2*>(a.gb + (int64_t)(k + u) * BS + kIPT * q);
        const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&raw.x);
        const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&raw.y);
        g[u][0] = __low2float(lo); g[u][1] = __high2float(lo);
        g[u][2] = __low2float(hi); g[u][3] = __high2float(hi);
      } else {
        const float gs = __bfloat162float(a.g[k + u]);
#pragma unroll
        for (int j = 0; j < kIPT; ++j) g[u][j] = gs;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      xv[u] = k + u < k1 ? X[(int64_t)c[u] * TPR + q] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < kIPT; ++j) acc[j] = fmaf(g[u][j], get4(xv[u], j), acc[j]);
  }
  return make_float4(acc[0], acc[1], acc[2], acc[3]);
}

// Row products of the kernel: shared-memory gathers (GU > 0) or registers.
// Every variant adds the entries of a row in the same order, so all give
// bit-identical results.
template <int GU>
__device__ __forceinline__ float4 edge_form4(const BatchArgs& a, int64_t i, int q,
                                             const int (&st)[kIPT], const float4* X) {
  if constexpr (GU > 0) return edge_form4_async<GU>(a, i, q, st, X);
  else return edge_form4_reg(a, i, q, st, X);
}
template <int GU>
__device__ __forceinline__ float4 fsai4(const BatchArgs& a, int64_t i, int q, bool lower,
                                        const float4* X) {
  if constexpr (GU > 0) return fsai4_async<GU>(a, i, q, lower, X);
  else return fsai4_reg(a, i, q, lower, X);
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

template <int GU>
__global__ void __launch_bounds__(kBBlock, 1)
pcg_batched_persistent(BatchArgs a) {
  // barrier test: bar[3] != 0 withholds the last block, so the others'
  // first barrier wait runs out (DEC_ERR_TIMEOUT)
  if (*(volatile unsigned*)(a.bar + 3) && blockIdx.x == gridDim.x - 1) return;
  __shared__ BState S;
  __shared__ double sh[kBBlock * kIPT];
  const int BS = a.BS, TPR = BS / kIPT;
  const int64_t n = a.n;
  const int q = threadIdx.x % TPR;                     // instance quad of this thread
  const int rpb = kBBlock / TPR;                       // rows per block and pass
  const int64_t row0 = (int64_t)blockIdx.x * rpb + threadIdx.x / TPR;
  const int64_t rstep = (int64_t)gridDim.x * rpb;
  const int64_t nq = n * TPR;                          // float4 elements of a vector
  const int64_t e0 = (int64_t)blockIdx.x * kBBlock + threadIdx.x;
  const int64_t estep = (int64_t)gridDim.x * kBBlock;
  int st[kIPT];
#pragma unroll
  for (int j = 0; j < kIPT; ++j) st[j] = a.states ? kIPT * q + j : 0;
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

  // ---- start: x64 = 0, r64 = b, r = (float) b, x = p = 0, |b|^2 per instance
  {
    double v[1][kIPT] = {{0.0, 0.0, 0.0, 0.0}};
    for (int64_t e = e0; e < nq; e += estep) {
      float4 rf;
#pragma unroll
      for (int j = 0; j < kIPT; ++j) {
        const double bi = a.bvec[e * kIPT + j];
        a.x64[e * kIPT + j] = 0.0;
        a.r64[e * kIPT + j] = bi;
        set4(rf, j, (float)bi);
        v[0][j] = fma(bi, bi, v[0][j]);
      }
      R[e] = rf;
      X[e] = make_float4(0.f, 0.f, 0.f, 0.f);
      Pv[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (!breduce<1>(v, a.partial, parity, S, sh, BS, a.bar, err)) return;
  }
  if (threadIdx.x < BS) {
    const int i = threadIdx.x;
    S.bnorm2[i] = S.red[0][i];
    S.best[i] = S.red[0][i];
    S.tol2[i] = a.seg2 * S.red[0][i];
    S.active[i] = (i < a.B && S.red[0][i] > 0.0) ? 1 : 0;
    S.iterating[i] = S.active[i];
    S.restart[i] = 1;
    S.stall[i] = 0;
    S.iters[i] = 0;
    S.rz[i] = 0.0;
  }
  __syncthreads();

  for (;;) {
    // ---- segment start for the active instances: z = M r, p = z + beta p
    if (any4(S.active))
      for (int64_t i = row0; i < n; i += rstep) T[i * TPR + q] = fsai4<GU>(a, i, q, true, R);
    if (!bgrid_sync(a.bar, err)) return;
    {
      Acc2 acc[kIPT];
      if (any4(S.active))
        for (int64_t i = row0; i < n; i += rstep) {
          const float4 zi = fsai4<GU>(a, i, q, false, T);
          Z[i * TPR + q] = zi;
          const float4 ri = R[i * TPR + q];
#pragma unroll
          for (int j = 0; j < kIPT; ++j) acc[j].add(get4(ri, j), get4(zi, j));
        }
      double v[1][kIPT];
#pragma unroll
      for (int j = 0; j < kIPT; ++j) v[0][j] = acc[j].get();
      if (!breduce<1>(v, a.partial, parity, S, sh, BS, a.bar, err)) return;
    }
    if (threadIdx.x < BS) {
      const int i = threadIdx.x;
      const double rzn = S.red[0][i];
      S.beta[i] = (S.restart[i] || S.rz[i] == 0.0) ? 0.0f : (float)(rzn / S.rz[i]);
      S.rz[i] = rzn;
      S.iterating[i] = S.active[i];
    }
    __syncthreads();
    if (any4(S.active)) {
      float4 bt;
#pragma unroll
      for (int j = 0; j < kIPT; ++j) set4(bt, j, S.beta[kIPT * q + j]);
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
          for (int64_t i = row0; i < n; i += rstep) {
            const float4 qi = edge_form4<GU>(a, i, q, st, Pv);
            Q[i * TPR + q] = qi;
            const float4 pi = Pv[i * TPR + q];
#pragma unroll
            for (int j = 0; j < kIPT; ++j) acc[j].add(get4(pi, j), get4(qi, j));
          }
        double v[1][kIPT];
#pragma unroll
        for (int j = 0; j < kIPT; ++j) v[0][j] = acc[j].get();
        if (!breduce<1>(v, a.partial, parity, S, sh, BS, a.bar, err)) return;
      }
      if (threadIdx.x < BS) {
        const int i = threadIdx.x;
        const double pq = S.red[0][i];
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
          float4 al;
#pragma unroll
          for (int j = 0; j < kIPT; ++j) set4(al, j, S.alpha[kIPT * q + j]);
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
        double v[1][kIPT];
#pragma unroll
        for (int j = 0; j < kIPT; ++j) v[0][j] = acc[j].get();
        if (!breduce<1>(v, a.partial, parity, S, sh, BS, a.bar, err)) return;
      }
      if (threadIdx.x < BS) {
        const int i = threadIdx.x;
        if (S.iterating[i]) {
          S.iters[i] += 1;
          const double rr = S.red[0][i];
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
      if (any4(S.iterating))
        for (int64_t i = row0; i < n; i += rstep) T[i * TPR + q] = fsai4<GU>(a, i, q, true, R);
      if (!bgrid_sync(a.bar, err)) return;
      {
        Acc2 acc[kIPT];
        if (any4(S.iterating))
          for (int64_t i = row0; i < n; i += rstep) {
            const float4 zi = fsai4<GU>(a, i, q, false, T);
            Z[i * TPR + q] = zi;
            const float4 ri = R[i * TPR + q];
#pragma unroll
            for (int j = 0; j < kIPT; ++j) acc[j].add(get4(ri, j), get4(zi, j));
          }
        double v[1][kIPT];
#pragma unroll
        for (int j = 0; j < kIPT; ++j) v[0][j] = acc[j].get();
        if (!breduce<1>(v, a.partial, parity, S, sh, BS, a.bar, err)) return;
      }
      if (threadIdx.x < BS) {
        const int i = threadIdx.x;
        if (S.iterating[i]) {
          S.beta[i] = (float)(S.red[0][i] / S.rz[i]);
          S.rz[i] = S.red[0][i];
        }
      }
      __syncthreads();
      if (any4(S.iterating)) {
        float4 bt;
        bool on[kIPT];
#pragma unroll
        for (int j = 0; j < kIPT; ++j) {
          set4(bt, j, S.beta[kIPT * q + j]);
          on[j] = act(S.iterating, j);
        }
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
      double v[1][kIPT] = {{0.0, 0.0, 0.0, 0.0}};
      if (any4(S.active))
        for (int64_t i = row0; i < n; i += rstep) {
          double y[kIPT];
          edge_form4_64(a, i, q, st, a.x64, y);
          float4 rf;
#pragma unroll
          for (int j = 0; j < kIPT; ++j) {
            const int64_t e = i * BS + kIPT * q + j;
            const double ri = a.bvec[e] - y[j];
            a.r64[e] = ri;
            set4(rf, j, (float)ri);
            v[0][j] = fma(ri, ri, v[0][j]);
          }
          R[i * TPR + q] = rf;
        }
      if (!breduce<1>(v, a.partial, parity, S, sh, BS, a.bar, err)) return;
    }
    if (threadIdx.x < BS) {
      const int i = threadIdx.x;
      if (S.active[i]) {
        const double rr = S.red[0][i];
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
// Per-instance FSAI factors for the batched solve (same definition as the
// single-instance factor: row i solves L_b[P_i, P_i] g = e_i and stores
// g / sqrt(g_i)), computed in FP32 from the edge form of L_b and stored in
// BF16 with the instances contiguous per entry.  A group of BS threads
// handles one row, thread b instance b, each with the packed lower triangle
// of its block in shared memory (k <= kBFsaiMax).  Longer rows (about 3 %
// of the rows at a limit of 12, which lets two blocks share an SM) keep the
// shared factor of the uncracked operator.
#ifndef DEC_BFSAI_MAX
#define DEC_BFSAI_MAX 12
#endif
constexpr int kBFsaiMax = DEC_BFSAI_MAX;
constexpr int kBFsaiTpb = 256;
constexpr int kBPacked = kBFsaiMax * (kBFsaiMax + 1) / 2;

__device__ __forceinline__ int btri(int r, int c) { return r * (r + 1) / 2 + c; }

__global__ void __launch_bounds__(kBFsaiTpb)
batch_fsai_kernel(int64_t n, int BS, int states, const int32_t* __restrict__ rowptr,
                  const int32_t* __restrict__ col, const int32_t* __restrict__ dpos,
                  const int32_t* __restrict__ eid, const int32_t* __restrict__ pos_up,
                  const uint8_t* __restrict__ tag, const float* __restrict__ w32,
                  const uint8_t* __restrict__ fc, const __nv_bfloat16* __restrict__ g0,
                  __nv_bfloat16* __restrict__ gb) {
  extern __shared__ float bsm[];
  float* A = bsm + threadIdx.x;                                  // stride kBFsaiTpb
  int32_t* P = reinterpret_cast<int32_t*>(bsm + kBPacked * kBFsaiTpb) + threadIdx.x;
  const int stride = kBFsaiTpb;
  const int b = threadIdx.x % BS;
  const int rpb = kBFsaiTpb / BS;
  const int state = states ? b : 0;
  for (int64_t i = (int64_t)blockIdx.x * rpb + threadIdx.x / BS; i < n;
       i += (int64_t)gridDim.x * rpb) {
    const int32_t k0 = rowptr[i], kd = dpos[i];
    const int k = kd - k0 + 1;
    if (k > kBFsaiMax) {   // this row's lower part and its transposed slots
      for (int32_t kk = k0; kk <= kd; ++kk) {
        gb[(int64_t)kk * BS + b] = g0[kk];
        if (kk < kd) gb[(int64_t)pos_up[eid[kk]] * BS + b] = g0[pos_up[eid[kk]]];
      }
      continue;
    }
    for (int q = 0; q < k; ++q) P[q * stride] = col[k0 + q];
    // gather L_b[P, P] (edge form; Dirichlet rows/columns eliminated)
    float dmax = 0.0f;
    for (int q = 0; q < k; ++q) {
      const int32_t r = P[q * stride];
      for (int c = 0; c < q; ++c) A[btri(q, c) * stride] = 0.0f;
      if (tag[r] == DEC_NODE_DIRICHLET) { A[btri(q, q) * stride] = 1.0f; dmax = fmaxf(dmax, 1.0f); continue; }
      float dsum = 0.0f;
      int c = 0;
      for (int32_t kk = rowptr[r]; kk < rowptr[r + 1]; ++kk) {
        const float m = (int)fc[kk] > state ? w32[kk] : 0.0f;
        dsum += m;
        const int32_t cc = col[kk];
        if (kk < dpos[r]) {            // lower part of row r: columns < r
          while (c < q && P[c * stride] < cc) ++c;
          if (c < q && P[c * stride] == cc && tag[cc] != DEC_NODE_DIRICHLET)
            A[btri(q, c) * stride] = -m;
        }
      }
      A[btri(q, q) * stride] = dsum == 0.0f ? 1.0f : dsum;
      dmax = fmaxf(dmax, A[btri(q, q) * stride]);
    }
    // Cholesky in place; a pivot <= 1e-6 max(diag) marks a singular block,
    // which is shifted by 1e-5 max(diag) and factored again
    bool ok = true;
    for (int pass = 0; pass < 2; ++pass) {
      ok = true;
      for (int c = 0; c < k && ok; ++c) {
        const float d = A[btri(c, c) * stride];
        if (!(d > (pass == 0 ? 1e-6f * dmax : 0.0f))) { ok = false; break; }
        const float lc = sqrtf(d), inv = 1.0f / lc;
        A[btri(c, c) * stride] = lc;
        for (int r = c + 1; r < k; ++r) A[btri(r, c) * stride] *= inv;
        for (int r = c + 1; r < k; ++r) {
          const float lrc = A[btri(r, c) * stride];
          for (int q = c + 1; q <= r; ++q) A[btri(r, q) * stride] -= lrc * A[btri(q, c) * stride];
        }
      }
      if (ok || pass == 1) break;
      // rebuild with a shift (the gather again, diagonal + shift)
      for (int q = 0; q < k; ++q) {
        const int32_t r = P[q * stride];
        for (int c = 0; c < q; ++c) A[btri(q, c) * stride] = 0.0f;
        if (tag[r] == DEC_NODE_DIRICHLET) { A[btri(q, q) * stride] = 1.0f + 1e-5f * dmax; continue; }
        float dsum = 0.0f;
        int c = 0;
        for (int32_t kk = rowptr[r]; kk < rowptr[r + 1]; ++kk) {
          const float m = (int)fc[kk] > state ? w32[kk] : 0.0f;
          dsum += m;
          const int32_t cc = col[kk];
          if (kk < dpos[r]) {
            while (c < q && P[c * stride] < cc) ++c;
            if (c < q && P[c * stride] == cc && tag[cc] != DEC_NODE_DIRICHLET)
              A[btri(q, c) * stride] = -m;
          }
        }
        A[btri(q, q) * stride] = (dsum == 0.0f ? 1.0f : dsum) + 1e-5f * dmax;
      }
    }
    // C^T g = e_k, g_j over the used diagonal slot
    for (int j = k - 1; j >= 0; --j) {
      float sum = (j == k - 1) ? 1.0f : 0.0f;
      for (int r = j + 1; r < k; ++r) sum -= A[btri(r, j) * stride] * A[btri(r, r) * stride];
      A[btri(j, j) * stride] = ok ? sum / A[btri(j, j) * stride] : 0.0f;
    }
    for (int q = 0; q < k; ++q) {
      const __nv_bfloat16 gq = ok ? __float2bfloat16_rn(A[btri(q, q) * stride]) : g0[k0 + q];
      gb[(int64_t)(k0 + q) * BS + b] = gq;
      if (q < k - 1) gb[(int64_t)pos_up[eid[k0 + q]] * BS + b] = gq;
    }
  }
}


// per-entry edge data for the edge form: *1 (FP32, FP64) and first crack
// state of the entry's edge; the diagonal slot gets w = 0, never cut
__global__ void batch_entries_kernel(int64_t nnz, const int32_t* __restrict__ eid,
                                     const double* __restrict__ w,
                                     const uint8_t* __restrict__ first_cut,
                                     float* __restrict__ w32, double* __restrict__ w64,
                                     uint8_t* __restrict__ fc, const double* __restrict__ g64,
                                     __nv_bfloat16* __restrict__ g16) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = eid[k];
    const double we = e >= 0 ? w[e] : 0.0;
    w32[k] = (float)we;
    w64[k] = we;
    fc[k] = e >= 0 ? first_cut[e] : (uint8_t)255;
    g16[k] = __float2bfloat16_rn((float)g64[k]);
  }
}

// right-hand sides b[i][inst] = sum over Dirichlet neighbours j of
// w_ij [inst < fc] T0_j (0 on Dirichlet rows and on rows all of whose
// weights are zero in that instance), the node form of Eq. 12
__global__ void batch_rhs_kernel(int64_t n, int B, int BS, int states, int sets,
                                 const int32_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ col,
                                 const int32_t* __restrict__ dpos,
                                 const uint8_t* __restrict__ tag,
                                 const double* __restrict__ w64,
                                 const uint8_t* __restrict__ fc,
                                 const double* __restrict__ T0, double* __restrict__ bvec) {
  const int64_t ne = n * BS;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / BS;
    const int inst = (int)(e % BS);
    double bi = 0.0;
    if (inst < B && tag[i] != DEC_NODE_DIRICHLET) {
      const int st = states ? inst : 0;
      const double* t0 = T0 + (sets ? (int64_t)inst * n : 0);
      double dsum = 0.0;
      for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        if (k == dpos[i]) continue;
        const double m = (int)fc[k] > st ? w64[k] : 0.0;
        dsum += m;
        if (tag[col[k]] == DEC_NODE_DIRICHLET) bi += m * t0[col[k]];
      }
      if (dsum == 0.0) bi = 0.0;
    }
    bvec[e] = bi;
  }
}

// rhs of every instance in the per-instance layout b[inst][i] (getters)
__global__ void batch_rhs_unpack_kernel(int64_t n, int B, int BS, const double* __restrict__ bb,
                                        double* __restrict__ b) {
  const int64_t total = n * B;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t inst = k / n, i = k % n;
    b[k] = bb[i * BS + inst];
  }
}

// u[inst][i] = x64[i][inst]
__global__ void batch_unpack_kernel(int64_t n, int B, int BS, const double* __restrict__ x64,
                                    double* __restrict__ u) {
  const int64_t total = n * B;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t inst = k / n, i = k % n;
    u[k] = x64[i * BS + inst];
  }
}

int batch_stride(int B) {
  int bs = 8;
  while (bs < B) bs <<= 1;
  return bs;
}

// Build the shared per-entry data, the BF16 factor copy and b[n][BS].
dec_status batch_setup(dec_ctx* ctx) {
  const int64_t n = ctx->n, nnz = ctx->nnz;
  cudaStream_t s = ctx->stream;
  const int B = ctx->B, BS = batch_stride(B);
  DEC_TRY(ctx->bw32.ensure(nnz));
  DEC_TRY(ctx->bw64.ensure(nnz));
  DEC_TRY(ctx->bfc.ensure(nnz));
  DEC_TRY(ctx->bg16.ensure(nnz));
  DEC_TRY(ctx->bb.ensure((size_t)n * BS));
  const unsigned g = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((nnz + 255) / 256, (int64_t)ctx->num_sms * 16));
  batch_entries_kernel<<<g, 256, 0, s>>>(nnz, ctx->eid.p, ctx->w.p, ctx->first_cut.p,
                                         ctx->bw32.p, ctx->bw64.p, ctx->bfc.p, ctx->g64.p,
                                         ctx->bg16.p);
  const unsigned g2 = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((n * BS + 255) / 256, (int64_t)ctx->num_sms * 16));
  batch_rhs_kernel<<<g2, 256, 0, s>>>(n, B, BS, ctx->n_scales > 1, ctx->n_sets > 1,
                                      ctx->rowptr.p, ctx->col.p, ctx->dpos.p, ctx->tag.p,
                                      ctx->bw64.p, ctx->bfc.p, ctx->T0.p, ctx->bb.p);
  const unsigned g3 = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((n * B + 255) / 256, (int64_t)ctx->num_sms * 16));
  batch_rhs_unpack_kernel<<<g3, 256, 0, s>>>(n, B, BS, ctx->bb.p, ctx->b.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 3;
  if (ctx->n_scales > 1) {
    // crack states change L per instance: one FSAI factor per state
    DEC_TRY(ctx->bgb.ensure((size_t)nnz * BS));
    const size_t smem = (size_t)kBPacked * kBFsaiTpb * sizeof(float) +
                        (size_t)kBFsaiMax * kBFsaiTpb * sizeof(int32_t);
    DEC_TRY(cudaFuncSetAttribute(batch_fsai_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    const int rpb = kBFsaiTpb / BS;
    const unsigned gf = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((n + rpb - 1) / rpb, (int64_t)ctx->num_sms * 8));
    batch_fsai_kernel<<<gf, kBFsaiTpb, smem, s>>>(
        n, BS, 1, ctx->rowptr.p, ctx->col.p, ctx->dpos.p, ctx->eid.p, ctx->pos_up.p,
        ctx->tag.p, ctx->bw32.p, ctx->bfc.p, ctx->bg16.p, ctx->bgb.p);
    DEC_TRY(cudaGetLastError());
    ctx->launches += 1;
    ctx->batch_per_instance = true;
  } else {
    ctx->batch_per_instance = false;   // Dirichlet sets share L and its factor
  }
  return DEC_OK;
}

dec_status solve_batched(dec_ctx* ctx, double rtol, int max_iter, int* iters,
                         double* relres) {
  const int64_t n = ctx->n;
  cudaStream_t s = ctx->stream;
  const int B = ctx->B, BS = batch_stride(B);
  if (B > kBMax) return ctx->fail(DEC_ERR_LIMIT, "batched solve: more than 64 instances");
  int coop = 0;
  DEC_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device));
  if (!coop) return ctx->fail(DEC_ERR_LIMIT, "batched solve: cooperative launch unavailable");
  const void* kern[kNumGatherVariants] = {
      (const void*)pcg_batched_persistent<0>, (const void*)pcg_batched_persistent<4>,
      (const void*)pcg_batched_persistent<6>, (const void*)pcg_batched_persistent<8>};
  const int smem[kNumGatherVariants] = {0, gather_smem<4>(), gather_smem<6>(), gather_smem<8>()};
  bool usable[kNumGatherVariants];
  bool any = false;
  for (int v = 0; v < kNumGatherVariants; ++v) {
    int per_sm = 0;
    DEC_TRY(cudaFuncSetAttribute(kern[v], cudaFuncAttributeMaxDynamicSharedMemorySize, smem[v]));
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
  DEC_TRY(ctx->bpartial.ensure((size_t)4 * grid * BS));
  DEC_TRY(ctx->coop.ensure(16 + 3 * kBMax));
  unsigned* bar = reinterpret_cast<unsigned*>(ctx->coop.p);
  int* status = reinterpret_cast<int*>(ctx->coop.p + 2);
  int* its = reinterpret_cast<int*>(ctx->coop.p + 16);
  double* result = reinterpret_cast<double*>(ctx->coop.p + 16 + kBMax / 2);
  BatchArgs a{};
  a.n = n;
  a.B = B;
  a.BS = BS;
  a.rowptr = ctx->rowptr.p;
  a.col = ctx->col.p;
  a.dpos = ctx->dpos.p;
  a.tag = ctx->tag.p;
  a.w32 = ctx->bw32.p;
  a.w64 = ctx->bw64.p;
  a.fc = ctx->bfc.p;
  a.states = ctx->n_scales > 1;
  a.g = ctx->bg16.p;
  a.gb = ctx->batch_per_instance ? ctx->bgb.p : nullptr;
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
    cudaError_t e = cudaMemsetAsync(ctx->coop.p, 0, sizeof(int64_t) * (16 + 3 * kBMax), s);
    if (e == cudaSuccess) e = write_barrier_test(ctx, bar);
    if (e == cudaSuccess)
      e = cudaLaunchCooperativeKernel(kern[v], dim3(grid), dim3(kBBlock), args, smem[v], s);
    ctx->launches += 1;
    return e;
  };
  // Autotuner: the first batched solve of a problem size at this instance
  // stride times kTuneIters FP32 iterations of every gather variant and keeps
  // the fastest (register gathers won at 8 instances, shared-memory gathers of 6
  // entries at 64).  All variants give bit-identical results.
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
  DEC_TRY(launch(v, max_iter));
  DEC_TRY(cudaEventRecord(k1, s));
  const unsigned g2 = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((n * B + 255) / 256, (int64_t)ctx->num_sms * 16));
  batch_unpack_kernel<<<g2, 256, 0, s>>>(n, B, BS, ctx->bx64.p, ctx->u.p);
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
