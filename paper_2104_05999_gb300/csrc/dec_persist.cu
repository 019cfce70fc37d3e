// dec_persist.cu - the mixed-precision PCG of one instance as a single
// persistent kernel (cooperative launch: every block is resident).
//
// The solve is the one of the mixed mode in dec_solver.cu: CG with FP32
// vectors and L, a BF16 FSAI factor (or FP32 Jacobi), and FP64 defect
// correction by reliable updates (x64 += x32, r = b - L x64 in FP64 each time
// the FP32 residual has dropped by 1e-2; convergence decided in FP64).  The
// phases of an iteration are separated by a grid barrier instead of kernel
// boundaries, and every reduction ends with all blocks summing the block
// partials in the same order, so each block holds the same alpha, beta and
// residuals and takes the same branch without a host round trip.
//
// The barrier spins on a generation counter with a bounded number of polls;
// when the bound is hit the kernel records DEC_ERR_TIMEOUT and every block
// leaves at its next barrier.  Words 2 and 3 of the barrier (zero in normal
// use) let a test shorten the bound and withhold a block, so that this
// failure path runs without any endless wait.
#include "dec_kern.cuh"

#include <algorithm>
#include <type_traits>

namespace dec {

constexpr long kSpinLimit = 1L << 24;   // polls of 32-256 ns: a few seconds
// One block of 1024 threads per SM: fewer blocks make the grid barrier and
// the all-blocks partial sums cheaper (they cost per block, not per thread).
constexpr int kPBlock = 1024;

struct PersistArgs {
  int64_t n;
  SellArg<float> A32;
  SellArg<double> A64;
  SellArg<__nv_bfloat16> Glo, Gup;
  const float* dinv;          // Jacobi, or nullptr for FSAI
  const double* b;
  double *x64, *r64;
  float *x, *r, *z, *p, *q, *t;
  float *r2, *p2;             // second buffers of r and p
  double* partial;            // [4][gridDim.x]
  unsigned* bar;              // [0] arrivals, [1] generation
  int* status;                // [0] error, [1] iterations, [2] outcome
  double* result;             // [0] final rr (FP64), [1] |b|^2
  double rtol2, seg2;
  int max_iter;
};

// Grid barrier with a bounded spin.  Returns false once any block has
// timed out (then every block leaves).
__device__ __forceinline__ bool grid_sync(unsigned* bar, int* err) {
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
      const long limit = lim ? (long)lim : kSpinLimit;
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

// Sum of NV (<= 2) per-thread values over the grid, identical in every
// block.  Consecutive calls alternate between two partial buffers: a block
// may write the partials of one sum while a slower block still reads those
// of the previous one, but never those of the one before (a barrier lies in
// between).  FP32 contributions (T = float) are added in FP32 inside each
// warp; everything above the warp level is FP64 and done by warp 0 alone
// (GB300's FP64 pipe is narrow, so FP64 work by every warp would dominate).
template <int NV, typename T>
__device__ __forceinline__ bool grid_sum(const T (&v)[NV], double (&tot)[NV],
                                         double* partial, int& parity, unsigned* bar,
                                         int* err) {
  __shared__ double sh[kPBlock];
  __shared__ double bc[2];
  double* part = partial + (size_t)parity * 2 * gridDim.x;
  parity ^= 1;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s;
    if constexpr (sizeof(T) == 4) s = block_sum_f<kPBlock>(v[k], sh);
    else s = block_sum<kPBlock>(v[k], sh);
    if (threadIdx.x == 0) part[k * gridDim.x + blockIdx.x] = s;
  }
  if (!grid_sync(bar, err)) return false;
  if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double t = warp0_sum_array(part + k * gridDim.x, (int)gridDim.x);
      if (threadIdx.x == 0) bc[k] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = bc[k];
  __syncthreads();
  return true;
}

// Row sum over the lane's row of slice s with the gathered operand formed on
// the fly: sum_j a_j * (X[c_j] + coef * Y[c_j]).  Used to fuse the vector
// update that produced the operand into the product that consumes it (the
// owner of row c computes the same fmaf for its own entry, so both agree).
template <typename MT>
__device__ __forceinline__ float sell_row2(const SellArg<MT>& A, int64_t s, int lane,
                                           const float* __restrict__ X,
                                           const float* __restrict__ Y, float coef) {
  constexpr int U = 8;
  const int32_t base = __ldg(A.sptr + s);
  const int32_t w = (__ldg(A.sptr + s + 1) - base) >> 5;
  const int32_t* __restrict__ cp = A.col + base + lane;
  const MT* __restrict__ vp = A.val + base + lane;
  float acc = 0.0f;
  for (int32_t j = 0; j < w; j += U) {
    int32_t c[U];
    MT av[U];
    float xv[U], yv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = j + u < w;
      c[u] = ok ? __ldg(cp + 32 * (j + u)) : 0;
      av[u] = ok ? vp[32 * (j + u)] : MT(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      xv[u] = j + u < w ? X[c[u]] : 0.0f;
      yv[u] = j + u < w ? Y[c[u]] : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j + u < w) acc = fma_(av[u], fmaf(coef, yv[u], xv[u]), acc);
  }
  return acc;
}

// One CG iteration is three phases separated by the three grid reductions
// it needs (p.q, r.r, r.z):
//   A: p_k = z + beta p_{k-1} (own rows) and q = L p_k, gathering z and
//      p_{k-1} so that p_k need not be complete first;
//   B: r_{k+1} = r_k - alpha q, x += alpha p_k (own rows) and t = G r_{k+1},
//      gathering r_k and q;
//   C: z = G^T t and r.z.
// p and r alternate between two buffers (a phase gathers the old vector while
// owners write the new one).  With Jacobi, B computes z = r / diag directly
// and C disappears.
template <bool JACOBI>
__global__ void __launch_bounds__(kPBlock, 1)
pcg_mixed_persistent(PersistArgs a) {
  // barrier test: bar[3] != 0 withholds the last block, so the others'
  // first barrier wait runs out (DEC_ERR_TIMEOUT)
  if (*(volatile unsigned*)(a.bar + 3) && blockIdx.x == gridDim.x - 1) return;
  const int64_t n = a.n;
  const int64_t gtid = blockIdx.x * (int64_t)kPBlock + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * kPBlock;
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = gtid >> 5, nwarps = gstride >> 5;
  int* err = a.status;
  __shared__ float s_scal;
  __shared__ int s_flag;
  auto finish = [&](int outcome, int iters, double rr, double bb) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.status[1] = iters;
      a.status[2] = outcome;
      a.result[0] = rr;
      a.result[1] = bb;
    }
  };
  float* P[2] = {a.p, a.p2};
  float* R[2] = {a.r, a.r2};
  int cur = 0;
  // one slice per warp at a time; the gathered operand is X[c] (+ coef *
  // Y[c] when Y is given).  (Interleaving two slices per warp needed more
  // than the 64 registers a 1024-thread block allows and ran slower.)
  auto slices = [&](const auto& A, auto&& body, const float* X, const float* Y, float coef) {
    for (int64_t s = gwarp; s < A.nslices; s += nwarps) {
      const float acc = Y ? sell_row2(A, s, lane, X, Y, coef) : sell_row(A, s, lane, X);
      const int32_t r0 = __ldg(A.perm + 32 * s + lane);
      if (r0 >= 0) body(r0, acc);
    }
  };

  // ---- start: x64 = 0, r64 = b, r = (float) b, x = p = 0
  int parity = 0;
  double v1[1], t1[1];
  {
    double bb = 0.0;
    for (int64_t i = gtid; i < n; i += gstride) {
      const double bi = a.b[i];
      a.x64[i] = 0.0;
      a.r64[i] = bi;
      a.r[i] = (float)bi;
      a.x[i] = 0.0f;
      a.p[i] = 0.0f;
      a.p2[i] = 0.0f;
      bb += bi * bi;
    }
    v1[0] = bb;
  }
  if (!grid_sum<1>(v1, t1, a.partial, parity, a.bar, err)) return;
  const double bnorm2 = t1[0];
  if (bnorm2 == 0.0) { finish(0, 0, 0.0, 0.0); return; }
  double rr64 = bnorm2, best = bnorm2, rz = 0.0;
  double tol2 = a.seg2 * rr64;
  int iters = 0, stall = 0, restart = 1;
  float beta = 0.0f;

  for (;;) {
    // ---- segment start: z = M r (from R[cur]), r.z, beta
    {
      float v[1] = {0.0f};
      double t[1];
      const float* rc = R[cur];
      if (JACOBI) {
        float acc = 0.0f;
        for (int64_t i = gtid; i < n; i += gstride) {
          const float zi = a.dinv[i] * rc[i];
          a.z[i] = zi;
          acc = fmaf(rc[i], zi, acc);
        }
        v[0] = acc;
      } else {
        slices(a.Glo, [&](int32_t row, float acc) { a.t[row] = acc; }, rc,
              (const float*)nullptr, 0.0f);
        if (!grid_sync(a.bar, err)) return;
        float acc2 = 0.0f;
        slices(a.Gup, [&](int32_t row, float acc) {
          a.z[row] = acc;
          acc2 = fmaf(rc[row], acc, acc2);
        }, a.t, (const float*)nullptr, 0.0f);
        v[0] = acc2;
      }
      if (!grid_sum<1>(v, t, a.partial, parity, a.bar, err)) return;
      if (threadIdx.x == 0) s_scal = (restart || rz == 0.0) ? 0.0f : (float)(t[0] / rz);
      __syncthreads();
      beta = s_scal;
      rz = t[0];
    }
    // ---- FP32 iterations until the residual has dropped by seg2
    int breakdown = 0;
    for (;;) {
      const int nxt = cur ^ 1;
      // A: p_k = z + beta p_{k-1}, q = L p_k, p_k . q
      {
        const float* pold = P[cur];
        float* pnew = P[nxt];
        float acc2 = 0.0f;
        slices(a.A32, [&](int32_t row, float qi) {
          const float pi = fmaf(beta, pold[row], a.z[row]);
          pnew[row] = pi;
          a.q[row] = qi;
          acc2 = fmaf(pi, qi, acc2);
        }, a.z, pold, beta);
        float vq[1] = {acc2};
        double tq[1];
        if (!grid_sum<1>(vq, tq, a.partial, parity, a.bar, err)) return;
        if (threadIdx.x == 0) {
          const double pq = tq[0];
          s_flag = (!(pq > 0.0) || !isfinite(pq)) ? 1 : 0;
          s_scal = s_flag ? 0.0f : (float)(rz / pq);
        }
        __syncthreads();
      }
      if (s_flag) { breakdown = 1; cur = nxt; break; }   // p_k is in P[nxt]
      const float alpha = s_scal;
      // B: r_{k+1} = r_k - alpha q, x += alpha p_k, t = G r_{k+1}, r.r
      float rr = 0.0f, rzj = 0.0f;
      {
        const float* rold = R[cur];
        float* rnew = R[nxt];
        const float* pk = P[nxt];
        if (JACOBI) {
          for (int64_t i = gtid; i < n; i += gstride) {
            const float ri = fmaf(-alpha, a.q[i], rold[i]);
            rnew[i] = ri;
            a.x[i] = fmaf(alpha, pk[i], a.x[i]);
            rr = fmaf(ri, ri, rr);
            const float zi = a.dinv[i] * ri;
            a.z[i] = zi;
            rzj = fmaf(ri, zi, rzj);
          }
        } else {
          slices(a.Glo, [&](int32_t row, float ti) {
            const float ri = fmaf(-alpha, a.q[row], rold[row]);
            rnew[row] = ri;
            a.x[row] = fmaf(alpha, pk[row], a.x[row]);
            a.t[row] = ti;
            rr = fmaf(ri, ri, rr);
          }, rold, (const float*)a.q, -alpha);
        }
      }
      float v2[2] = {rr, rzj};
      double t2[2];
      if (!grid_sum<2>(v2, t2, a.partial, parity, a.bar, err)) return;
      cur = nxt;
      ++iters;
      if (t2[0] <= tol2 || iters >= a.max_iter || !isfinite(t2[0])) break;
      double rz_new;
      if (JACOBI) {
        rz_new = t2[1];
      } else {
        // C: z = G^T t, r.z
        float acc2 = 0.0f;
        const float* rcur = R[cur];
        slices(a.Gup, [&](int32_t row, float zi) {
          a.z[row] = zi;
          acc2 = fmaf(rcur[row], zi, acc2);
        }, a.t, (const float*)nullptr, 0.0f);
        float vz[1] = {acc2};
        double tz[1];
        if (!grid_sum<1>(vz, tz, a.partial, parity, a.bar, err)) return;
        rz_new = tz[0];
      }
      if (threadIdx.x == 0) s_scal = (float)(rz_new / rz);
      __syncthreads();
      beta = s_scal;
      rz = rz_new;
    }
    // ---- reliable update: x64 += x, x = 0; r64 = b - L x64; R[cur] = (float) r64
    for (int64_t i = gtid; i < n; i += gstride) {
      a.x64[i] += (double)a.x[i];
      a.x[i] = 0.0f;
    }
    if (!grid_sync(a.bar, err)) return;
    {
      double rr = 0.0;
      float* rc = R[cur];
      for (int64_t s = gwarp; s < a.A64.nslices; s += nwarps) {
        const int32_t row = __ldg(a.A64.perm + 32 * s + lane);
        const double acc = sell_row(a.A64, s, lane, a.x64);
        if (row >= 0) {
          const double ri = a.b[row] - acc;
          a.r64[row] = ri;
          rc[row] = (float)ri;
          rr = fma(ri, ri, rr);
        }
      }
      v1[0] = rr;
    }
    if (!grid_sum<1>(v1, t1, a.partial, parity, a.bar, err)) return;
    rr64 = t1[0];
    if (rr64 <= a.rtol2 * bnorm2) { finish(0, iters, rr64, bnorm2); return; }
    if (iters >= a.max_iter) { finish(1, iters, rr64, bnorm2); return; }
    if (rr64 < 0.5 * best) { best = rr64; stall = 0; }
    else if (++stall >= 4) { finish(2, iters, rr64, bnorm2); return; }
    restart = (breakdown || stall > 0) ? 1 : 0;
    tol2 = a.seg2 * rr64;
  }
}

// One mixed-precision solve of instance `inst` with the persistent kernel.
// Returns DEC_ERR_LIMIT when a cooperative launch is not possible (the
// caller then uses the kernel-per-phase path).
dec_status solve_mixed_persistent(dec_ctx* ctx, int inst, double rtol, int max_iter,
                                  int* iters_out, double* relres_out) {
  const int64_t n = ctx->n;
  const int vs = value_set(ctx, inst);
  cudaStream_t s = ctx->stream;
  const bool fsai = ctx->precond == DEC_PRECOND_FSAI;
  int dev_coop = 0;
  DEC_TRY(cudaDeviceGetAttribute(&dev_coop, cudaDevAttrCooperativeLaunch, ctx->device));
  if (!dev_coop) return DEC_ERR_LIMIT;
  auto kern = fsai ? pcg_mixed_persistent<false> : pcg_mixed_persistent<true>;
  int per_sm = 0;
  DEC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPBlock, 0));
  if (per_sm < 1) return DEC_ERR_LIMIT;
  const int grid = ctx->num_sms;   // one block per SM (per_sm >= 1 checked)
  DEC_TRY(ctx->partial.ensure((size_t)kRedSlots * std::max(grid, ctx->reduce_grid)));
  DEC_TRY(ctx->coop.ensure(16));
  unsigned* bar = reinterpret_cast<unsigned*>(ctx->coop.p);
  int* status = reinterpret_cast<int*>(ctx->coop.p + 2);
  double* result = reinterpret_cast<double*>(ctx->coop.p + 8);
  DEC_TRY(cudaMemsetAsync(ctx->coop.p, 0, 16 * sizeof(int64_t), s));
  DEC_TRY(write_barrier_test(ctx, bar));
  PersistArgs a{};
  a.n = n;
  a.A32 = sell_arg(ctx->sellL, ctx->sL32.p + (int64_t)vs * ctx->sellL.total);
  a.A64 = sell_arg(ctx->sellL, ctx->sL64.p + (int64_t)vs * ctx->sellL.total);
  a.Glo = sell_arg(ctx->sellLo, fsai ? ctx->sGlo16.p + (int64_t)vs * ctx->sellLo.total : nullptr);
  a.Gup = sell_arg(ctx->sellUp, fsai ? ctx->sGup16.p + (int64_t)vs * ctx->sellUp.total : nullptr);
  a.dinv = fsai ? nullptr : ctx->dinv32.p + (int64_t)vs * n;
  a.b = ctx->b.p + (int64_t)inst * n;
  a.x64 = ctx->u.p + (int64_t)inst * n;
  a.r64 = ctx->r64.p;
  a.x = ctx->x32.p; a.r = ctx->r32.p; a.z = ctx->z32.p; a.p = ctx->p32.p;
  a.q = ctx->q32.p; a.t = ctx->t32.p;
  DEC_TRY(ctx->r32b.ensure(n));
  DEC_TRY(ctx->p32b.ensure(n));
  a.r2 = ctx->r32b.p; a.p2 = ctx->p32b.p;
  a.partial = ctx->partial.p;
  a.bar = bar;
  a.status = status;
  a.result = result;
  a.rtol2 = rtol * rtol;
  a.seg2 = 1e-4;
  a.max_iter = max_iter;
  void* args[] = {&a};
  DEC_TRY(cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(kPBlock), args, 0, s));
  ctx->launches += 1;
  int hs[3];
  double hr[2];
  DEC_TRY(cudaMemcpyAsync(hs, status, sizeof(hs), cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaMemcpyAsync(hr, result, sizeof(hr), cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaStreamSynchronize(s));
  *iters_out = hs[1];
  *relres_out = hr[1] > 0.0 ? std::sqrt(hr[0] / hr[1]) : 0.0;
  if (hs[0]) return ctx->fail(DEC_ERR_TIMEOUT, "persistent solve: a grid barrier timed out");
  if (hs[2] == 1) return ctx->fail(DEC_NOT_CONVERGED, "max_iter reached");
  if (hs[2] == 2) return ctx->fail(DEC_NOT_CONVERGED, "residual replacement stalled");
  return DEC_OK;
}

}  // namespace dec
