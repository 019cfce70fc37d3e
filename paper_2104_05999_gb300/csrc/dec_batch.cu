// dec_batch.cu - many instances on one mesh in one persistent launch: the
// crack states of a growing disc population (each state zeroes the *1 of the
// edges it cuts, Sec. 2.5) or several Dirichlet value sets, solved together
// by mixed-precision PCG over a sparse matrix - multiple vector product.
//
// The instances share L's sparsity; vectors are stored node-major with the
// instances contiguous (X[i * BS + b], BS = padded instance count), so one
// gathered neighbour row X[c][0..BS) is one coalesced load.  A group of BS
// threads works on one row, thread b on instance b.  The operator of
// instance b is applied in "edge form" from shared per-entry data (column,
// *1 in FP32 and FP64, first crack state):
//   (L_b x)_i = sum_k w_k [b < fc_k] (x_i - x_c),
// which needs no per-instance values or diagonal (vectors are zero on
// Dirichlet nodes, so those columns drop out; Dirichlet rows and rows whose
// weights are all zero in instance b are identity rows).  All instances use
// one FSAI factor, that of the uncracked operator.
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
      long polls = 0;
      unsigned ns = 32;
      while (*gen == g) {
        if (++polls > kBSpinLimit || *(volatile int*)err) {
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

// Per-instance grid reduction of NV values; thread t contributes v[k] to
// instance t % BS.  Results land in S.red[k][b], identical in every block.
template <int NV>
__device__ bool breduce(const double (&v)[NV], double* partial, int& parity, BState& S,
                        double* sh, int BS, unsigned* bar, int* err) {
  const int G = gridDim.x;
  double* part = partial + (size_t)parity * 2 * G * BS;
  parity ^= 1;
  const int per = kBBlock / BS;            // threads per instance in a block
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    sh[threadIdx.x] = v[k];
    __syncthreads();
    if (threadIdx.x < BS) {
      double s = 0.0;
      for (int j = 0; j < per; ++j) s += sh[threadIdx.x + j * BS];
      part[((size_t)k * G + blockIdx.x) * BS + threadIdx.x] = s;
    }
    __syncthreads();
  }
  if (!bgrid_sync(bar, err)) return false;
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

// y = L_b x for row i, instance b; FP32 (T = float) or FP64.  Entries are
// taken 8 at a time (8 column/weight/state loads, then 8 independent
// gathers) to keep loads in flight.  The diagonal slot carries w = 0, so it
// needs no test.
template <typename T>
__device__ __forceinline__ T edge_form_row(const BatchArgs& a, int64_t i, int b, int state,
                                           const T* __restrict__ X, const T* __restrict__ w) {
  constexpr int U = 8;
  const int32_t k0 = a.rowptr[i], k1 = a.rowptr[i + 1];
  const int BS = a.BS;
  const T xi = X[i * BS + b];
  if (a.tag[i] == DEC_NODE_DIRICHLET) return xi;
  T acc = T(0), dsum = T(0);
  for (int32_t k = k0; k < k1; k += U) {
    int32_t c[U];
    T m[U], xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = k + u < k1;
      c[u] = ok ? __ldg(a.col + k + u) : 0;
      const T wk = ok ? __ldg(w + k + u) : T(0);
      const int f = ok ? (int)__ldg(a.fc + k + u) : 0;
      m[u] = f > state ? wk : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = k + u < k1 ? X[(int64_t)c[u] * BS + b] : T(0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      dsum += m[u];
      acc += m[u] * xv[u];
    }
  }
  return dsum == T(0) ? xi : dsum * xi - acc;
}

// FSAI halves with the shared factor (lower: G, upper: G^T), 8 at a time
__device__ __forceinline__ float fsai_row(const BatchArgs& a, int64_t i, int b, bool lower,
                                          const float* __restrict__ X) {
  constexpr int U = 8;
  const int32_t k0 = lower ? a.rowptr[i] : a.dpos[i];
  const int32_t k1 = lower ? a.dpos[i] + 1 : a.rowptr[i + 1];
  const int BS = a.BS;
  float acc = 0.0f;
  for (int32_t k = k0; k < k1; k += U) {
    int32_t c[U];
    float g[U], xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = k + u < k1;
      c[u] = ok ? __ldg(a.col + k + u) : 0;
      g[u] = !ok ? 0.0f
                 : __bfloat162float(a.gb ? a.gb[(int64_t)(k + u) * BS + b] : a.g[k + u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = k + u < k1 ? X[(int64_t)c[u] * BS + b] : 0.0f;
#pragma unroll
    for (int u = 0; u < U; ++u) acc = fmaf(g[u], xv[u], acc);
  }
  return acc;
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

__global__ void __launch_bounds__(kBBlock, 1)
pcg_batched_persistent(BatchArgs a) {
  __shared__ BState S;
  __shared__ double sh[kBBlock];
  const int BS = a.BS;
  const int64_t n = a.n;
  const int b = threadIdx.x % BS;                       // this thread's instance
  const int rpb = kBBlock / BS;                         // rows per block and pass
  const int64_t row0 = (int64_t)blockIdx.x * rpb + threadIdx.x / BS;
  const int64_t rstep = (int64_t)gridDim.x * rpb;
  const int64_t ne = n * BS;
  const int64_t e0 = (int64_t)blockIdx.x * kBBlock + threadIdx.x;
  const int64_t estep = (int64_t)gridDim.x * kBBlock;
  const int state = a.states ? b : 0;
  int* err = a.status;
  int parity = 0;

  // ---- start: x64 = 0, r64 = b, r = (float) b, x = p = 0, |b|^2 per instance
  {
    double bb = 0.0;
    for (int64_t e = e0; e < ne; e += estep) {
      const double bi = a.bvec[e];
      a.x64[e] = 0.0;
      a.r64[e] = bi;
      a.r[e] = (float)bi;
      a.x[e] = 0.0f;
      a.p[e] = 0.0f;
      bb = fma(bi, bi, bb);
    }
    double v[1] = {bb};
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
    for (int64_t i = row0; i < n; i += rstep)
      if (S.active[b]) a.t[i * BS + b] = fsai_row(a, i, b, true, a.r);
    if (!bgrid_sync(a.bar, err)) return;
    {
      Acc2 rz;
      for (int64_t i = row0; i < n; i += rstep)
        if (S.active[b]) {
          const float zi = fsai_row(a, i, b, false, a.t);
          a.z[i * BS + b] = zi;
          rz.add(a.r[i * BS + b], zi);
        }
      double v[1] = {rz.get()};
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
    for (int64_t e = e0; e < ne; e += estep)
      if (S.active[b]) a.p[e] = fmaf(S.beta[b], a.p[e], a.z[e]);
    if (!bgrid_sync(a.bar, err)) return;

    // ---- FP32 iterations until every working instance is frozen
    for (;;) {
      {
        Acc2 pq;
        for (int64_t i = row0; i < n; i += rstep)
          if (S.iterating[b]) {
            const float qi = edge_form_row<float>(a, i, b, state, a.p, a.w32);
            a.q[i * BS + b] = qi;
            pq.add(a.p[i * BS + b], qi);
          }
        double v[1] = {pq.get()};
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
        Acc2 rr;
        for (int64_t e = e0; e < ne; e += estep)
          if (S.iterating[b]) {
            const float al = S.alpha[b];
            const float ri = fmaf(-al, a.q[e], a.r[e]);
            a.x[e] = fmaf(al, a.p[e], a.x[e]);
            a.r[e] = ri;
            rr.add(ri, ri);
          }
        double v[1] = {rr.get()};
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
      for (int64_t i = row0; i < n; i += rstep)
        if (S.iterating[b]) a.t[i * BS + b] = fsai_row(a, i, b, true, a.r);
      if (!bgrid_sync(a.bar, err)) return;
      {
        Acc2 rz;
        for (int64_t i = row0; i < n; i += rstep)
          if (S.iterating[b]) {
            const float zi = fsai_row(a, i, b, false, a.t);
            a.z[i * BS + b] = zi;
            rz.add(a.r[i * BS + b], zi);
          }
        double v[1] = {rz.get()};
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
      for (int64_t e = e0; e < ne; e += estep)
        if (S.iterating[b]) a.p[e] = fmaf(S.beta[b], a.p[e], a.z[e]);
      if (!bgrid_sync(a.bar, err)) return;
    }

    // ---- reliable update of the active instances
    for (int64_t e = e0; e < ne; e += estep)
      if (S.active[b]) {
        a.x64[e] += (double)a.x[e];
        a.x[e] = 0.0f;
      }
    if (!bgrid_sync(a.bar, err)) return;
    {
      double rr = 0.0;
      for (int64_t i = row0; i < n; i += rstep)
        if (S.active[b]) {
          const int64_t e = i * BS + b;
          const double ri = a.bvec[e] - edge_form_row<double>(a, i, b, state, a.x64, a.w64);
          a.r64[e] = ri;
          a.r[e] = (float)ri;
          rr = fma(ri, ri, rr);
        }
      double v[1] = {rr};
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
// of its block in shared memory (k <= kBFsaiMax).  Longer rows keep the
// shared factor of the uncracked operator.
constexpr int kBFsaiMax = 16;
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
  int coop = 0, per_sm = 0;
  DEC_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device));
  DEC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_batched_persistent,
                                                        kBBlock, 0));
  if (!coop || per_sm < 1)
    return ctx->fail(DEC_ERR_LIMIT, "batched solve: cooperative launch unavailable");
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
  DEC_TRY(cudaMemsetAsync(ctx->coop.p, 0, sizeof(int64_t) * (16 + 3 * kBMax), s));
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
  DEC_TRY(cudaLaunchCooperativeKernel((const void*)pcg_batched_persistent, dim3(grid),
                                      dim3(kBBlock), args, 0, s));
  ctx->launches += 1;
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
