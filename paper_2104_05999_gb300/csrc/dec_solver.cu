// dec_solver.cu - preconditioned conjugate gradients on the node Laplacian
// (the Krylov solve of Sec. 2.3, stopped at a relative residual as in
// Sec. 3.1) and the effective conductivity from the boundary flux (Sec. 2.5).
//
// Every iteration runs as a few memory-bound kernels that keep all scalars
// (alpha, beta, r.z, ...) in device memory; dot products are reduced inside
// the producing kernel (block partials, the last block finishes in a fixed
// order), so results are deterministic and the host only polls a `done`
// flag once per chunk of iterations.  A chunk is captured once into a CUDA
// graph and replayed.
//
//   FP64 mode : x, r, z, p, q in FP64; L and the preconditioner in FP64.
//   mixed mode: FP64 defect correction r = b - L x around an inner PCG whose
//               vectors and L are FP32 and whose FSAI factor is BF16 (or an
//               FP32 Jacobi); x += e after every inner solve.
#include "dec_internal.cuh"

#include <algorithm>
#include <cmath>

namespace dec {

__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T> struct Acc;           // row accumulation type
template <> struct Acc<double> { using type = double; };
template <> struct Acc<float> { using type = float; };

template <typename VT, typename MT>
__device__ __forceinline__ VT mul_acc(VT acc, MT a, VT x);
template <> __device__ __forceinline__ double mul_acc(double acc, double a, double x) { return fma(a, x, acc); }
template <> __device__ __forceinline__ float mul_acc(float acc, float a, float x) { return fmaf(a, x, acc); }
template <> __device__ __forceinline__ float mul_acc(float acc, __nv_bfloat16 a, float x) { return fmaf(__bfloat162float(a), x, acc); }
template <> __device__ __forceinline__ double mul_acc(double acc, __nv_bfloat16 a, double x) { return fma((double)__bfloat162float(a), x, acc); }

// Sum over entries k in [k0, k1) of a[k] * x[col[k]] by a group of TPR lanes;
// the total is returned in every lane of the group.
template <int TPR, typename MT, typename VT>
__device__ __forceinline__ VT row_sum(int lir, int32_t k0, int32_t k1,
                                      const int32_t* __restrict__ col,
                                      const MT* __restrict__ a,
                                      const VT* __restrict__ x) {
  VT s = VT(0);
  for (int32_t k = k0 + lir; k < k1; k += TPR) s = mul_acc(s, a[k], __ldg(x + col[k]));
#pragma unroll
  for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, TPR);
  return s;
}

// ------------------------------------------------------------ kernels
// Launch shape of the vector kernels: fixed grid (reduce_grid blocks of
// kBlock threads), grid-stride over rows.

template <typename BT, typename VT>
__global__ void __launch_bounds__(kBlock)
cg_init_kernel(int64_t n, const BT* __restrict__ b, VT* __restrict__ x,
               VT* __restrict__ r, VT* __restrict__ p, double rtol2,
               CgScalars* cg, double* partial, unsigned* ticket) {
  double bb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    VT bi = (VT)b[i];
    x[i] = VT(0);
    r[i] = bi;
    p[i] = VT(0);
    bb += to_d(bi) * to_d(bi);
  }
  double v[1] = {bb}, t[1];
  if (grid_reduce<kBlock, 1>(v, t, partial, ticket) && threadIdx.x == 0) {
    cg->bnorm2 = t[0];
    cg->tol2 = rtol2 * t[0];
    cg->rr = t[0];
    cg->done = t[0] == 0.0 ? 1 : 0;
    cg->iters = 0;
    cg->breakdown = 0;
    cg->beta = 0.0;
    cg->rz = 0.0;
  }
}

// q = A p and alpha = (r.z) / (p.q)
template <int TPR, typename MT, typename VT>
__global__ void __launch_bounds__(kBlock)
spmv_pq_kernel(int64_t n, const int32_t* __restrict__ rowptr,
               const int32_t* __restrict__ col, const MT* __restrict__ val,
               const VT* __restrict__ p, VT* __restrict__ q, CgScalars* cg,
               double* partial, unsigned* ticket) {
  if (*(volatile int*)&cg->done) return;
  const int lir = threadIdx.x % TPR;
  const int64_t groups = (int64_t)gridDim.x * (kBlock / TPR);
  double pq = 0.0;
  // all lanes of a group run the same number of loop trips (n rounded up)
  for (int64_t i = blockIdx.x * (int64_t)(kBlock / TPR) + threadIdx.x / TPR;
       i - (int64_t)(threadIdx.x / TPR) < n; i += groups) {
    const bool ok = i < n;
    const int32_t k0 = ok ? rowptr[i] : 0, k1 = ok ? rowptr[i + 1] : 0;
    VT s = row_sum<TPR>(lir, k0, k1, col, val, p);
    if (ok && lir == 0) {
      q[i] = s;
      pq += to_d(p[i]) * to_d(s);
    }
  }
  double v[1] = {pq}, t[1];
  if (grid_reduce<kBlock, 1>(v, t, partial, ticket) && threadIdx.x == 0) {
    const double den = t[0];
    if (!(den > 0.0) || !isfinite(den)) {
      cg->breakdown = 1;
      cg->done = 1;
      cg->alpha = 0.0;
    } else {
      cg->pq = den;
      cg->alpha = cg->rz / den;
    }
  }
}

// x += alpha p, r -= alpha q, r.r; with Jacobi also z = dinv r and r.z
template <typename VT, typename DT, bool JACOBI>
__global__ void __launch_bounds__(kBlock)
update_kernel(int64_t n, VT* __restrict__ x, VT* __restrict__ r,
              const VT* __restrict__ p, const VT* __restrict__ q,
              const DT* __restrict__ dinv, VT* __restrict__ z, int max_iter,
              CgScalars* cg, double* partial, unsigned* ticket) {
  if (*(volatile int*)&cg->done) return;
  const VT alpha = (VT)cg->alpha;
  double rr = 0.0, rz = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    VT xi = x[i] + alpha * p[i];
    VT ri = r[i] - alpha * q[i];
    x[i] = xi;
    r[i] = ri;
    rr += to_d(ri) * to_d(ri);
    if (JACOBI) {
      VT zi = (VT)dinv[i] * ri;
      z[i] = zi;
      rz += to_d(ri) * to_d(zi);
    }
  }
  double v[2] = {rr, rz}, t[2];
  if (grid_reduce<kBlock, 2>(v, t, partial, ticket) && threadIdx.x == 0) {
    cg->rr = t[0];
    cg->iters += 1;
    if (t[0] <= cg->tol2 || cg->iters >= max_iter || !isfinite(t[0])) cg->done = 1;
    if (JACOBI) {
      cg->beta = t[1] / cg->rz;
      cg->rz = t[1];
    }
  }
}

// FSAI apply, first half: t = G r over entries up to the diagonal
template <int TPR, typename PT, typename VT>
__global__ void __launch_bounds__(kBlock)
fsai_lower_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                  const int32_t* __restrict__ dpos, const int32_t* __restrict__ col,
                  const PT* __restrict__ g, const VT* __restrict__ r,
                  VT* __restrict__ t, const CgScalars* cg) {
  if (*(volatile const int*)&cg->done) return;
  const int lir = threadIdx.x % TPR;
  const int64_t groups = (int64_t)gridDim.x * (kBlock / TPR);
  for (int64_t i = blockIdx.x * (int64_t)(kBlock / TPR) + threadIdx.x / TPR;
       i - (int64_t)(threadIdx.x / TPR) < n; i += groups) {
    const bool ok = i < n;
    const int32_t k0 = ok ? rowptr[i] : 0, k1 = ok ? dpos[i] + 1 : 0;
    VT s = row_sum<TPR>(lir, k0, k1, col, g, r);
    if (ok && lir == 0) t[i] = s;
  }
}

// FSAI apply, second half: z = G^T t over entries from the diagonal on,
// r.z, then beta = (r.z)_new / (r.z)_old.  `init` keeps beta = 0.
template <int TPR, typename PT, typename VT>
__global__ void __launch_bounds__(kBlock)
fsai_upper_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                  const int32_t* __restrict__ dpos, const int32_t* __restrict__ col,
                  const PT* __restrict__ g, const VT* __restrict__ t,
                  const VT* __restrict__ r, VT* __restrict__ z, int init,
                  CgScalars* cg, double* partial, unsigned* ticket) {
  if (*(volatile int*)&cg->done) return;
  const int lir = threadIdx.x % TPR;
  const int64_t groups = (int64_t)gridDim.x * (kBlock / TPR);
  double rz = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)(kBlock / TPR) + threadIdx.x / TPR;
       i - (int64_t)(threadIdx.x / TPR) < n; i += groups) {
    const bool ok = i < n;
    const int32_t k0 = ok ? dpos[i] : 0, k1 = ok ? rowptr[i + 1] : 0;
    VT s = row_sum<TPR>(lir, k0, k1, col, g, t);
    if (ok && lir == 0) {
      z[i] = s;
      rz += to_d(r[i]) * to_d(s);
    }
  }
  double v[1] = {rz}, tt[1];
  if (grid_reduce<kBlock, 1>(v, tt, partial, ticket) && threadIdx.x == 0) {
    cg->beta = init ? 0.0 : tt[0] / cg->rz;
    cg->rz = tt[0];
  }
}

// Jacobi at (re)start: z = dinv r, r.z
template <typename VT, typename DT>
__global__ void __launch_bounds__(kBlock)
jacobi_init_kernel(int64_t n, const DT* __restrict__ dinv, const VT* __restrict__ r,
                   VT* __restrict__ z, CgScalars* cg, double* partial,
                   unsigned* ticket) {
  if (*(volatile int*)&cg->done) return;
  double rz = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    VT zi = (VT)dinv[i] * r[i];
    z[i] = zi;
    rz += to_d(r[i]) * to_d(zi);
  }
  double v[1] = {rz}, t[1];
  if (grid_reduce<kBlock, 1>(v, t, partial, ticket) && threadIdx.x == 0) {
    cg->beta = 0.0;
    cg->rz = t[0];
  }
}

// p = z + beta p
template <typename VT>
__global__ void __launch_bounds__(kBlock)
xpay_kernel(int64_t n, const VT* __restrict__ z, VT* __restrict__ p,
            const CgScalars* cg) {
  if (*(volatile const int*)&cg->done) return;
  const VT beta = (VT)cg->beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// FP64 residual r = b - A x, r.r into *out; optionally r32 = (float) r
template <int TPR>
__global__ void __launch_bounds__(kBlock)
residual_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                const int32_t* __restrict__ col, const double* __restrict__ val,
                const double* __restrict__ x, const double* __restrict__ b,
                double* __restrict__ r, float* __restrict__ r32, double* out,
                double* partial, unsigned* ticket) {
  const int lir = threadIdx.x % TPR;
  const int64_t groups = (int64_t)gridDim.x * (kBlock / TPR);
  double rr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)(kBlock / TPR) + threadIdx.x / TPR;
       i - (int64_t)(threadIdx.x / TPR) < n; i += groups) {
    const bool ok = i < n;
    const int32_t k0 = ok ? rowptr[i] : 0, k1 = ok ? rowptr[i + 1] : 0;
    double s = row_sum<TPR>(lir, k0, k1, col, val, x);
    if (ok && lir == 0) {
      double ri = b[i] - s;
      r[i] = ri;
      if (r32) r32[i] = (float)ri;
      rr += ri * ri;
    }
  }
  double v[1] = {rr}, t[1];
  if (grid_reduce<kBlock, 1>(v, t, partial, ticket) && threadIdx.x == 0) *out = t[0];
}

// x64 += e32
__global__ void __launch_bounds__(kBlock)
correct_kernel(int64_t n, double* __restrict__ x, const float* __restrict__ e) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] += (double)e[i];
}

// T = u + T0 on Dirichlet nodes
__global__ void __launch_bounds__(kBlock)
form_T_kernel(int64_t n, const double* __restrict__ u, const double* __restrict__ T0,
              const uint8_t* __restrict__ tag, double* __restrict__ T) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    T[i] = u[i] + (tag[i] == DEC_NODE_DIRICHLET ? T0[i] : 0.0);
}

// k_eff pieces (Sec. 2.5): net outflow sum_j w_ij (T_i - T_j) of Dirichlet
// nodes on x = 0 (q_in) and inflow on x = 1 (q_out), and the energy
// sum over edges of w_e (T_i - T_j)^2, all with the unmodified weights.
__global__ void __launch_bounds__(kBlock)
k_eff_kernel(int64_t n, const int32_t* __restrict__ rowptr,
             const int32_t* __restrict__ col, const int32_t* __restrict__ eid,
             const int32_t* __restrict__ dpos, const uint8_t* __restrict__ tag,
             const double* __restrict__ xyz, const double* __restrict__ w,
             const uint8_t* __restrict__ fc, int state, const double* __restrict__ T,
             double* out3, double* partial, unsigned* ticket) {
  double qin = 0.0, qout = 0.0, en = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double Ti = T[i];
    const int32_t k0 = rowptr[i], k1 = rowptr[i + 1], kd = dpos[i];
    double net = 0.0;
    for (int32_t k = k0; k < k1; ++k) {
      if (k == kd) continue;
      const int32_t e = eid[k];
      const double we = (int)fc[e] > state ? w[e] : 0.0;
      const double d = Ti - T[col[k]];
      net += we * d;
      if (k > kd) en += we * d * d;
    }
    if (tag[i] == DEC_NODE_DIRICHLET) {
      const double xi = xyz[3 * i];
      if (xi == 0.0) qin += net;
      else if (xi == 1.0) qout -= net;
    }
  }
  double v[3] = {qin, qout, en}, t[3];
  if (grid_reduce<kBlock, 3>(v, t, partial, ticket) && threadIdx.x == 0) {
    out3[0] = t[0];
    out3[1] = t[1];
    out3[2] = t[2];
  }
}

// ------------------------------------------------------------- driver
constexpr int kTpr = 8;          // lanes per CSR row (rows average ~16 nnz)
constexpr int kTprHalf = 4;      // lanes per half row (FSAI factor)
constexpr int kChunk = 16;       // iterations per graph launch / host poll

struct Bufs {
  // one precision's PCG vectors
  void *x, *r, *z, *p, *q, *t;
};

template <typename VT, typename MT, typename PT, typename DT>
static void launch_iterations(dec_ctx* ctx, int64_t n, const MT* val,
                              const PT* g, const DT* dinv, VT* x, VT* r, VT* z,
                              VT* p, VT* q, VT* t, int max_iter, int count) {
  cudaStream_t s = ctx->stream;
  const unsigned G = (unsigned)ctx->reduce_grid;
  CgScalars* cg = ctx->cg.p;
  double* part = ctx->partial.p;
  unsigned* tk = ctx->ticket.p;
  const bool jac = ctx->precond == DEC_PRECOND_JACOBI;
  ctx->launches += (int64_t)count * (jac ? 3 : 5);
  for (int it = 0; it < count; ++it) {
    spmv_pq_kernel<kTpr, MT, VT><<<G, kBlock, 0, s>>>(n, ctx->rowptr.p, ctx->col.p,
                                                     val, p, q, cg, part, tk);
    if (jac) {
      update_kernel<VT, DT, true><<<G, kBlock, 0, s>>>(n, x, r, p, q, dinv, z,
                                                       max_iter, cg, part, tk);
    } else {
      update_kernel<VT, DT, false><<<G, kBlock, 0, s>>>(n, x, r, p, q, dinv, z,
                                                        max_iter, cg, part, tk);
      fsai_lower_kernel<kTprHalf, PT, VT><<<G, kBlock, 0, s>>>(
          n, ctx->rowptr.p, ctx->dpos.p, ctx->col.p, g, r, t, cg);
      fsai_upper_kernel<kTprHalf, PT, VT><<<G, kBlock, 0, s>>>(
          n, ctx->rowptr.p, ctx->dpos.p, ctx->col.p, g, t, r, z, 0, cg, part, tk);
    }
    xpay_kernel<VT><<<G, kBlock, 0, s>>>(n, z, p, cg);
  }
}

// (Re)start: given r, compute z = M r, r.z, and p = z.
template <typename VT, typename PT, typename DT>
static void launch_restart(dec_ctx* ctx, int64_t n, const PT* g, const DT* dinv,
                           VT* r, VT* z, VT* p, VT* t) {
  cudaStream_t s = ctx->stream;
  const unsigned G = (unsigned)ctx->reduce_grid;
  CgScalars* cg = ctx->cg.p;
  ctx->launches += ctx->precond == DEC_PRECOND_JACOBI ? 2 : 3;
  if (ctx->precond == DEC_PRECOND_JACOBI) {
    jacobi_init_kernel<VT, DT><<<G, kBlock, 0, s>>>(n, dinv, r, z, cg, ctx->partial.p,
                                                    ctx->ticket.p);
  } else {
    fsai_lower_kernel<kTprHalf, PT, VT><<<G, kBlock, 0, s>>>(
        n, ctx->rowptr.p, ctx->dpos.p, ctx->col.p, g, r, t, cg);
    fsai_upper_kernel<kTprHalf, PT, VT><<<G, kBlock, 0, s>>>(
        n, ctx->rowptr.p, ctx->dpos.p, ctx->col.p, g, t, r, z, 1, cg,
        ctx->partial.p, ctx->ticket.p);
  }
  xpay_kernel<VT><<<G, kBlock, 0, s>>>(n, z, p, cg);
}

static dec_status read_cg(dec_ctx* ctx, CgScalars* h) {
  DEC_TRY(cudaMemcpyAsync(h, ctx->cg.p, sizeof(CgScalars), cudaMemcpyDeviceToHost,
                          ctx->stream));
  DEC_TRY(cudaStreamSynchronize(ctx->stream));
  return DEC_OK;
}

// Run chunks of iterations (one captured graph per chunk) until `done`.
template <typename VT, typename MT, typename PT, typename DT>
static dec_status run_pcg(dec_ctx* ctx, int64_t n, const MT* val, const PT* g,
                          const DT* dinv, VT* x, VT* r, VT* z, VT* p, VT* q, VT* t,
                          int max_iter, CgScalars* h) {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  DEC_TRY(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  launch_iterations<VT, MT, PT, DT>(ctx, n, val, g, dinv, x, r, z, p, q, t, max_iter,
                                    kChunk);
  cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
  if (ce != cudaSuccess) return ctx->cuda_fail(ce, "cudaStreamEndCapture");
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return ctx->cuda_fail(ce, "cudaGraphInstantiate");
  dec_status st = DEC_OK;
  const int64_t per_chunk = (int64_t)kChunk * (ctx->precond == DEC_PRECOND_JACOBI ? 3 : 5);
  ctx->launches -= per_chunk;  // capture itself launches nothing
  for (;;) {
    ctx->launches += per_chunk;
    ce = cudaGraphLaunch(exec, ctx->stream);
    if (ce != cudaSuccess) { st = ctx->cuda_fail(ce, "cudaGraphLaunch"); break; }
    st = read_cg(ctx, h);
    if (st != DEC_OK || h->done) break;
  }
  cudaGraphExecDestroy(exec);
  return st;
}

dec_status solve_instance(dec_ctx* ctx, int inst, double rtol, int max_iter,
                          int mode, int* iters_out, double* relres_out) {
  const int64_t n = ctx->n, nnz = ctx->nnz;
  const int vs = ctx->n_scales > 1 ? inst : 0;
  cudaStream_t s = ctx->stream;
  const unsigned G = (unsigned)ctx->reduce_grid;
  const double* val64 = ctx->val64.p + (int64_t)vs * nnz;
  const double* bvec = ctx->b.p + (int64_t)inst * n;
  double* u = ctx->u.p + (int64_t)inst * n;
  CgScalars h{};
  double* rr_dev = ctx->out3.p + 3 * (int64_t)ctx->B;  // scratch scalar
  double rr_true = 0.0, bnorm2 = 0.0;
  int total_iters = 0;
  dec_status st = DEC_OK;

  if (mode == DEC_MODE_FP64) {
    const double* g = ctx->g64.p + (int64_t)vs * nnz;
    const double* dinv = ctx->dinv64.p + (int64_t)vs * n;
    double *x = ctx->x64.p, *r = ctx->r64.p, *z = ctx->z64.p, *p = ctx->p64.p,
           *q = ctx->q64.p, *t = ctx->t64.p;
    ctx->launches += 1;
    cg_init_kernel<double, double><<<G, kBlock, 0, s>>>(n, bvec, x, r, p, rtol * rtol,
                                                        ctx->cg.p, ctx->partial.p,
                                                        ctx->ticket.p);
    launch_restart<double, double, double>(ctx, n, g, dinv, r, z, p, t);
    DEC_TRY(cudaGetLastError());
    for (;;) {
      st = run_pcg<double, double, double, double>(ctx, n, val64, g, dinv, x, r, z, p,
                                                   q, t, max_iter, &h);
      if (st != DEC_OK) return st;
      bnorm2 = h.bnorm2;
      total_iters = h.iters;
      if (bnorm2 == 0.0) { rr_true = 0.0; break; }
      // true residual, replacing the recursive one
      ctx->launches += 1;
      residual_kernel<kTpr><<<G, kBlock, 0, s>>>(n, ctx->rowptr.p, ctx->col.p, val64,
                                                x, bvec, r, nullptr, rr_dev,
                                                ctx->partial.p, ctx->ticket.p);
      DEC_TRY(cudaMemcpyAsync(&rr_true, rr_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
      DEC_TRY(cudaStreamSynchronize(s));
      if (h.breakdown) { st = ctx->fail(DEC_ERR_BREAKDOWN, "CG breakdown: p.Lp <= 0 or not finite"); break; }
      if (rr_true <= rtol * rtol * bnorm2) break;
      if (h.iters >= max_iter) { st = ctx->fail(DEC_NOT_CONVERGED, "max_iter reached"); break; }
      // restart from the true residual
      int zero = 0;
      DEC_TRY(cudaMemcpyAsync(&ctx->cg.p->done, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
      launch_restart<double, double, double>(ctx, n, g, dinv, r, z, p, t);
      DEC_TRY(cudaGetLastError());
    }
    DEC_TRY(cudaMemcpyAsync(u, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  } else {
    // mixed: FP64 defect correction around FP32 PCG
    const float* val32 = ctx->val32.p + (int64_t)vs * nnz;
    const __nv_bfloat16* g = ctx->g16.p + (int64_t)vs * nnz;
    const float* dinv = ctx->dinv32.p + (int64_t)vs * n;
    double* x64 = ctx->x64.p;
    double* r64 = ctx->r64.p;
    float *x = ctx->x32.p, *r = ctx->r32.p, *z = ctx->z32.p, *p = ctx->p32.p,
          *q = ctx->q32.p, *t = ctx->t32.p;
    DEC_TRY(cudaMemsetAsync(x64, 0, sizeof(double) * n, s));
    // r64 = b - L*0 = b, r32 = (float) b, |b|^2
    ctx->launches += 1;
    residual_kernel<kTpr><<<G, kBlock, 0, s>>>(n, ctx->rowptr.p, ctx->col.p, val64, x64,
                                              bvec, r64, ctx->t32.p, rr_dev,
                                              ctx->partial.p, ctx->ticket.p);
    DEC_TRY(cudaMemcpyAsync(&bnorm2, rr_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    DEC_TRY(cudaStreamSynchronize(s));
    rr_true = bnorm2;
    const double inner_rtol = 1e-4;
    double best = rr_true;
    int stall = 0;
    while (bnorm2 > 0.0 && rr_true > rtol * rtol * bnorm2) {
      if (total_iters >= max_iter) { st = ctx->fail(DEC_NOT_CONVERGED, "max_iter reached"); break; }
      ctx->launches += 3;  // init, correction, residual
      cg_init_kernel<float, float><<<G, kBlock, 0, s>>>(n, ctx->t32.p, x, r, p,
                                                        inner_rtol * inner_rtol,
                                                        ctx->cg.p, ctx->partial.p,
                                                        ctx->ticket.p);
      launch_restart<float, __nv_bfloat16, float>(ctx, n, g, dinv, r, z, p, t);
      DEC_TRY(cudaGetLastError());
      st = run_pcg<float, float, __nv_bfloat16, float>(ctx, n, val32, g, dinv, x, r, z,
                                                       p, q, t, max_iter - total_iters, &h);
      if (st != DEC_OK) return st;
      total_iters += h.iters;
      correct_kernel<<<G, kBlock, 0, s>>>(n, x64, x);
      residual_kernel<kTpr><<<G, kBlock, 0, s>>>(n, ctx->rowptr.p, ctx->col.p, val64,
                                                x64, bvec, r64, ctx->t32.p, rr_dev,
                                                ctx->partial.p, ctx->ticket.p);
      DEC_TRY(cudaMemcpyAsync(&rr_true, rr_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
      DEC_TRY(cudaStreamSynchronize(s));
      if (h.breakdown && !(rr_true < best)) {
        st = ctx->fail(DEC_ERR_BREAKDOWN, "CG breakdown in the FP32 inner solve");
        break;
      }
      if (rr_true < 0.25 * best) { best = rr_true; stall = 0; }
      else if (++stall >= 3) { st = ctx->fail(DEC_NOT_CONVERGED, "defect correction stalled"); break; }
    }
    DEC_TRY(cudaMemcpyAsync(u, x64, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  *iters_out = total_iters;
  *relres_out = bnorm2 > 0.0 ? std::sqrt(rr_true / bnorm2) : 0.0;
  return st;
}

dec_status k_eff_instance(dec_ctx* ctx, int inst, double* out3_host) {
  const int64_t n = ctx->n;
  cudaStream_t s = ctx->stream;
  const unsigned G = (unsigned)ctx->reduce_grid;
  const int ts = ctx->n_sets > 1 ? inst : 0;
  double* T = ctx->t64.p;  // scratch
  ctx->launches += 2;
  form_T_kernel<<<G, kBlock, 0, s>>>(n, ctx->u.p + (int64_t)inst * n,
                                     ctx->T0.p + (int64_t)ts * n, ctx->tag.p, T);
  k_eff_kernel<<<G, kBlock, 0, s>>>(n, ctx->rowptr.p, ctx->col.p, ctx->eid.p,
                                    ctx->dpos.p, ctx->tag.p, ctx->xyz.p, ctx->w.p,
                                    ctx->first_cut.p, ctx->n_scales > 1 ? inst : 0, T,
                                    ctx->out3.p + 3 * (int64_t)inst, ctx->partial.p,
                                    ctx->ticket.p);
  DEC_TRY(cudaGetLastError());
  DEC_TRY(cudaMemcpyAsync(out3_host, ctx->out3.p + 3 * (int64_t)inst,
                          3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaStreamSynchronize(s));
  return DEC_OK;
}

dec_status form_T(dec_ctx* ctx, int inst, double* T) {
  const int ts = ctx->n_sets > 1 ? inst : 0;
  ctx->launches += 1;
  form_T_kernel<<<(unsigned)ctx->reduce_grid, kBlock, 0, ctx->stream>>>(
      ctx->n, ctx->u.p + (int64_t)inst * ctx->n, ctx->T0.p + (int64_t)ts * ctx->n,
      ctx->tag.p, T);
  DEC_TRY(cudaGetLastError());
  return DEC_OK;
}

}  // namespace dec

namespace dec {

// Time `reps` launches of one solver kernel on the current instance's data,
// each preceded (outside the timed events) by a write of `flush_bytes` to
// evict L2, so the figure is the HBM-bound duration of a launch.
dec_status time_kernel(dec_ctx* ctx, int which, int reps, size_t flush_bytes,
                       double* avg_ms) {
  const int64_t n = ctx->n;
  cudaStream_t s = ctx->stream;
  const unsigned G = (unsigned)ctx->reduce_grid;
  DEC_TRY(ctx->flush.ensure(flush_bytes > 0 ? flush_bytes : 1));
  for (auto* bf : {&ctx->p64, &ctx->q64, &ctx->t64, &ctx->z64}) DEC_TRY(bf->ensure(n));
  for (auto* bf : {&ctx->p32, &ctx->q32, &ctx->t32, &ctx->z32, &ctx->r32}) DEC_TRY(bf->ensure(n));
  DEC_TRY(ctx->r64.ensure(n));
  // finite operands: p = b (and its FP32 copy), done = 0
  DEC_TRY(cudaMemcpyAsync(ctx->p64.p, ctx->b.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  DEC_TRY(cudaMemcpyAsync(ctx->r64.p, ctx->b.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  DEC_TRY(cudaMemsetAsync(ctx->p32.p, 0, sizeof(float) * n, s));
  DEC_TRY(cudaMemsetAsync(ctx->r32.p, 0, sizeof(float) * n, s));
  CgScalars h{};
  h.rz = 1.0;
  DEC_TRY(cudaMemcpyAsync(ctx->cg.p, &h, sizeof(h), cudaMemcpyHostToDevice, s));
  cudaEvent_t e0, e1;
  DEC_TRY(cudaEventCreate(&e0));
  DEC_TRY(cudaEventCreate(&e1));
  double total = 0.0;
  for (int it = 0; it < reps; ++it) {
    if (flush_bytes) DEC_TRY(cudaMemsetAsync(ctx->flush.p, it & 0xff, flush_bytes, s));
    DEC_TRY(cudaMemcpyAsync(&ctx->cg.p->done, &h.done, sizeof(int), cudaMemcpyHostToDevice, s));
    DEC_TRY(cudaEventRecord(e0, s));
    switch (which) {
      case DEC_KERNEL_SPMV_F64:
        spmv_pq_kernel<kTpr, double, double><<<G, kBlock, 0, s>>>(
            n, ctx->rowptr.p, ctx->col.p, ctx->val64.p, ctx->p64.p, ctx->q64.p, ctx->cg.p,
            ctx->partial.p, ctx->ticket.p);
        break;
      case DEC_KERNEL_SPMV_F32:
        spmv_pq_kernel<kTpr, float, float><<<G, kBlock, 0, s>>>(
            n, ctx->rowptr.p, ctx->col.p, ctx->val32.p, ctx->p32.p, ctx->q32.p, ctx->cg.p,
            ctx->partial.p, ctx->ticket.p);
        break;
      case DEC_KERNEL_FSAI_F64:
        fsai_lower_kernel<kTprHalf, double, double><<<G, kBlock, 0, s>>>(
            n, ctx->rowptr.p, ctx->dpos.p, ctx->col.p, ctx->g64.p, ctx->r64.p, ctx->t64.p, ctx->cg.p);
        fsai_upper_kernel<kTprHalf, double, double><<<G, kBlock, 0, s>>>(
            n, ctx->rowptr.p, ctx->dpos.p, ctx->col.p, ctx->g64.p, ctx->t64.p, ctx->r64.p,
            ctx->z64.p, 1, ctx->cg.p, ctx->partial.p, ctx->ticket.p);
        break;
      case DEC_KERNEL_FSAI_BF16:
        fsai_lower_kernel<kTprHalf, __nv_bfloat16, float><<<G, kBlock, 0, s>>>(
            n, ctx->rowptr.p, ctx->dpos.p, ctx->col.p, ctx->g16.p, ctx->r32.p, ctx->t32.p, ctx->cg.p);
        fsai_upper_kernel<kTprHalf, __nv_bfloat16, float><<<G, kBlock, 0, s>>>(
            n, ctx->rowptr.p, ctx->dpos.p, ctx->col.p, ctx->g16.p, ctx->t32.p, ctx->r32.p,
            ctx->z32.p, 1, ctx->cg.p, ctx->partial.p, ctx->ticket.p);
        break;
      default:
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return ctx->fail(DEC_ERR_ARG, "time_kernel: unknown kernel id");
    }
    DEC_TRY(cudaEventRecord(e1, s));
    DEC_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    DEC_TRY(cudaEventElapsedTime(&ms, e0, e1));
    total += ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *avg_ms = total / reps;
  return DEC_OK;
}

}  // namespace dec
