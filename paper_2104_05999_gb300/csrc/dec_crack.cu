// dec_crack.cu - crack growth (Sec. 2.5): one more dual face becomes
// insulating at every step and the steady solution and k_eff are computed
// again.  The deterministic rule of Sec. 3.3 cracks the face that carries
// the largest heat flux in the current solution; the stochastic rule of
// Sec. 3.4 cracks faces in a random order the caller draws.
//
// In the node form a dual face belongs to a primal edge e and its flux is
// the value of the flux 2-form on it, |w_e (T_i - T_j)|.  Every edge that
// still conducts (w_e > 0, not cut) is a candidate: each dual face lies
// between the dual cells of two nodes, the counterpart of the paper's
// non-boundary faces.  A crack marks the edge as cut in crack state 0, so
// L, b, the preconditioner and k_eff all see w_e = 0 from then on.
//
// A crack changes only a few values of the system (Sec. 2.3): rows and
// columns i, j of L, b_i, b_j, and the FSAI rows whose principal block holds
// i or j.  Each step updates just those and starts the solve from the
// previous solution; DEC_CRACK_REBUILD rebuilds everything and solves from
// zero instead.
#include "dec_internal.cuh"

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

namespace dec {

constexpr int kCrackBlock = 256;

// (value, edge) order of the pick: larger flux first, then smaller edge id
__device__ __forceinline__ bool crack_better(double v, int64_t e, double bv, int64_t be) {
  return v > bv || (v == bv && e < be);
}

__device__ __forceinline__ void crack_block_best(double& v, int64_t& e) {
  __shared__ double sv[kCrackBlock];
  __shared__ int64_t se[kCrackBlock];
  sv[threadIdx.x] = v;
  se[threadIdx.x] = e;
  __syncthreads();
  for (int h = kCrackBlock / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h &&
        crack_better(sv[threadIdx.x + h], se[threadIdx.x + h], sv[threadIdx.x], se[threadIdx.x])) {
      sv[threadIdx.x] = sv[threadIdx.x + h];
      se[threadIdx.x] = se[threadIdx.x + h];
    }
    __syncthreads();
  }
  v = sv[0];
  e = se[0];
}

// Best candidate of each block: flux |w_e (T_i - T_j)| of the conducting,
// uncut edges (fc = 0 means cut in state 0).
__global__ void __launch_bounds__(kCrackBlock)
crack_flux_best_kernel(int64_t ne, const int32_t* __restrict__ E, const double* __restrict__ w,
                       const uint8_t* __restrict__ fc, const double* __restrict__ T,
                       double* __restrict__ bval, int64_t* __restrict__ bidx) {
  double best = -1.0;
  int64_t be = INT64_MAX;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double we = fc[e] > 0 ? w[e] : 0.0;
    if (!(we > 0.0)) continue;
    const double f = fabs(we * (T[E[2 * e]] - T[E[2 * e + 1]]));
    if (crack_better(f, e, best, be)) {
      best = f;
      be = e;
    }
  }
  crack_block_best(best, be);
  if (threadIdx.x == 0) {
    bval[blockIdx.x] = best;
    bidx[blockIdx.x] = be;
  }
}

// One block: the best of the block bests; cracks it and records its id
// (-1 when no edge conducts any more).
__global__ void __launch_bounds__(kCrackBlock)
crack_pick_kernel(int nb, const double* __restrict__ bval, const int64_t* __restrict__ bidx,
                  uint8_t* __restrict__ fc, int64_t* __restrict__ picked) {
  double best = -1.0;
  int64_t be = INT64_MAX;
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    if (bidx[b] != INT64_MAX && crack_better(bval[b], bidx[b], best, be)) {
      best = bval[b];
      be = bidx[b];
    }
  crack_block_best(best, be);
  if (threadIdx.x == 0) {
    if (be == INT64_MAX) {
      *picked = -1;
    } else {
      fc[be] = 0;
      *picked = be;
    }
  }
}

// Ordered rule: crack edge e if it is a conducting, uncut edge; -2 otherwise.
__global__ void crack_take_kernel(int64_t e, int64_t ne, const double* __restrict__ w,
                                  uint8_t* __restrict__ fc, int64_t* __restrict__ picked) {
  if (e < 0 || e >= ne || !(w[e] > 0.0) || fc[e] == 0) {
    *picked = -2;
  } else {
    fc[e] = 0;
    *picked = e;
  }
}

dec_status crack_evolve(dec_ctx* ctx, int rule, int max_steps, const int32_t* order_host,
                        double rtol, int max_iter, int mode, double k_stop, int32_t* cracked,
                        double* k_eff, int32_t* steps) {
  cudaStream_t s = ctx->stream;
  const int64_t ne = ctx->ne;
  const unsigned G = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((ne + kCrackBlock - 1) / kCrackBlock, (int64_t)ctx->num_sms * 8));
  DEC_TRY(ctx->crack_buf.ensure((size_t)G + 1));
  DEC_TRY(ctx->t64.ensure(ctx->n));
  int64_t* bidx = ctx->crack_buf.p;
  int64_t* picked = ctx->crack_buf.p + G;
  double* bval = ctx->partial.p;   // capacity >= 8 blocks per SM
  *steps = 0;
  int it = 0;
  int64_t iters_total = 0;
  double rr = 0.0, o[3];
  // rule bit DEC_CRACK_REBUILD: rebuild L and the preconditioner and solve
  // from zero at every step (the reference behaviour); otherwise update the
  // rows a crack changes and start each solve from the previous solution
  const bool rebuild = (rule & DEC_CRACK_REBUILD) != 0;
  rule &= ~DEC_CRACK_REBUILD;
  auto solve = [&](bool warm) -> dec_status {
    dec_status st = solve_instance(ctx, 0, rtol, max_iter, mode, &it, &rr, warm);
    if (st != DEC_OK) return st;
    DEC_TRY_STATUS(form_T(ctx, 0, ctx->t64.p));   // T for the next pick
    return k_eff_all(ctx, o);                     // as dec_k_eff reports it
  };
  DEC_TRY_STATUS(solve(false));
  const double k0 = o[0];
  for (int step = 0; step < max_steps; ++step) {
    if (rule == DEC_CRACK_MAX_FLUX) {
      crack_flux_best_kernel<<<G, kCrackBlock, 0, s>>>(ne, ctx->E.p, ctx->w.p,
                                                       ctx->first_cut.p, ctx->t64.p, bval, bidx);
      crack_pick_kernel<<<1, kCrackBlock, 0, s>>>((int)G, bval, bidx, ctx->first_cut.p, picked);
      ctx->launches += 2;
    } else {
      crack_take_kernel<<<1, 1, 0, s>>>(order_host[step], ne, ctx->w.p, ctx->first_cut.p, picked);
      ctx->launches += 1;
    }
    DEC_TRY(cudaGetLastError());
    int64_t e = -1;
    DEC_TRY(cudaMemcpyAsync(&e, picked, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    DEC_TRY(cudaStreamSynchronize(s));
    if (e == -2)
      return ctx->fail(DEC_ERR_ARG, "crack_evolve: order[" + std::to_string(step) +
                                        "] is not a conducting, uncut edge");
    if (e < 0) break;   // nothing conducts any more
    if (rebuild) {
      DEC_TRY_STATUS(build_values(ctx, 0));
      DEC_TRY_STATUS(build_precond(ctx, 0));
    } else {
      DEC_TRY_STATUS(crack_update(ctx, e));
    }
    DEC_TRY_STATUS(solve(!rebuild));
    iters_total += it;
    cracked[step] = (int32_t)e;
    k_eff[step] = o[0];
    *steps = step + 1;
    if (o[0] <= k_stop * k0) break;
  }
  ctx->crack_iters = iters_total;
  return DEC_OK;
}

// ------------------------------------------------ Monte-Carlo paths
// Stochastic cracking (Sec. 3.4) of several paths at once: path b cracks
// the edges of its own caller-drawn order, one per step, in its own copy of
// *1 (w[b][e] = 0).  The paths are the instances of one batched solve, each
// step started from the previous solutions.

// Crack edge order[b][step] of every active path; an entry that is not a
// conducting, uncut edge of its path sets *bad = path + 1.
__global__ void crack_paths_take_kernel(int P, int step, int max_steps,
                                        const int32_t* __restrict__ orders,
                                        const uint8_t* __restrict__ active, int64_t ne,
                                        double* __restrict__ w, const uint8_t* __restrict__ fc,
                                        int* __restrict__ bad) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= P || !active[b]) return;
  const int64_t e = orders[(int64_t)b * max_steps + step];
  if (e < 0 || e >= ne || !(w[(int64_t)b * ne + e] > 0.0) || fc[e] == 0) {
    atomicMax(bad, b + 1);
    return;
  }
  w[(int64_t)b * ne + e] = 0.0;
}

dec_status crack_paths(dec_ctx* ctx, int P, int max_steps, const int32_t* orders_dev,
                       double rtol, int max_iter, double k_stop, double* k_eff,
                       int32_t* steps) {
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n, ne = ctx->ne;
  // P copies of the current *1 (field 0), one per path
  DEC_TRY(cudaStreamSynchronize(s));
  DEC_TRY(ctx->w.grow_keep((size_t)P * ne, ne));
  for (int b = 1; b < P; ++b)
    DEC_TRY(cudaMemcpyAsync(ctx->w.p + (int64_t)b * ne, ctx->w.p, sizeof(double) * ne,
                            cudaMemcpyDeviceToDevice, s));
  ctx->n_fields = P;
  ctx->B = P;
  ctx->precond = DEC_PRECOND_FSAI_SHARED;
  DEC_TRY(ctx->b.ensure((size_t)P * n));
  DEC_TRY(ctx->u.ensure((size_t)P * n));
  DEC_TRY(ctx->out3.ensure(3 * (size_t)P + 2));
  // the shared FSAI factor (kept by long rows) needs its buffers even when
  // the context was built with Jacobi
  DEC_TRY(ctx->g64.ensure(ctx->nnz));
  DEC_TRY(ctx->sGlo64.ensure(ctx->sellLo.total));
  DEC_TRY(ctx->sGup64.ensure(ctx->sellUp.total));
  DEC_TRY(ctx->sGlo16.ensure(ctx->sellLo.total));
  DEC_TRY(ctx->sGup16.ensure(ctx->sellUp.total));
  DEC_TRY_STATUS(build_values(ctx, 0));
  DEC_TRY_STATUS(build_precond(ctx, 0));   // the factor long rows keep
  DEC_TRY_STATUS(batch_setup(ctx));
  std::vector<int> it(P);
  std::vector<double> rr(P), o(3 * (size_t)P), k0(P);
  std::vector<uint8_t> act(P, 1);
  dec_status st = solve_batched(ctx, rtol, max_iter, it.data(), rr.data(), false);
  if (st != DEC_OK) return st;
  DEC_TRY_STATUS(k_eff_all(ctx, o.data()));
  for (int b = 0; b < P; ++b) {
    k0[b] = o[3 * b];
    steps[b] = 0;
  }
  DEC_TRY(ctx->crack_buf.ensure(((size_t)P + 15) / 8 + 2));
  uint8_t* d_act = reinterpret_cast<uint8_t*>(ctx->crack_buf.p + 1);
  int* d_bad = reinterpret_cast<int*>(ctx->crack_buf.p);
  int64_t iters_total = 0;
  for (int step = 0; step < max_steps; ++step) {
    int live = 0;
    for (int b = 0; b < P; ++b) live += act[b];
    if (!live) break;
    DEC_TRY(cudaMemcpyAsync(d_act, act.data(), P, cudaMemcpyHostToDevice, s));
    DEC_TRY(cudaMemsetAsync(d_bad, 0, sizeof(int), s));
    crack_paths_take_kernel<<<(P + 63) / 64, 64, 0, s>>>(P, step, max_steps, orders_dev, d_act,
                                                       ne, ctx->w.p, ctx->first_cut.p, d_bad);
    DEC_TRY(cudaGetLastError());
    ctx->launches += 1;
    int bad = 0;
    DEC_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    DEC_TRY(cudaStreamSynchronize(s));
    if (bad)
      return ctx->fail(DEC_ERR_ARG, "crack_paths: orders[" + std::to_string(bad - 1) + "][" +
                                        std::to_string(step) +
                                        "] is not a conducting, uncut edge of its path");
    DEC_TRY_STATUS(batch_refresh_values(ctx));
    st = solve_batched(ctx, rtol, max_iter, it.data(), rr.data(), true);
    if (st != DEC_OK) return st;
    for (int b = 0; b < P; ++b) iters_total += it[b];
    DEC_TRY_STATUS(k_eff_all(ctx, o.data()));
    for (int b = 0; b < P; ++b) {
      if (!act[b]) continue;
      k_eff[(int64_t)b * max_steps + step] = o[3 * b];
      steps[b] = step + 1;
      if (o[3 * b] <= k_stop * k0[b]) act[b] = 0;
    }
  }
  ctx->crack_iters = iters_total;
  return DEC_OK;
}

}  // namespace dec
