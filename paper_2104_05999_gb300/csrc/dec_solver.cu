// dec_solver.cu - preconditioned conjugate gradients on the node Laplacian
// (the Krylov solve of Sec. 2.3, stopped at a relative residual as in
// Sec. 3.1) and the effective conductivity from the boundary flux (Sec. 2.5).
//
// Every iteration runs as a few memory-bound kernels that keep all scalars
// (alpha, beta, r.z, ...) in device memory; dot products are reduced inside
// the producing kernel (block partials, the last block finishes in a fixed
// order), so results are deterministic and the host only polls a `done`
// flag once per chunk of iterations.  A chunk is captured once into a CUDA
// graph and replayed.  Matrix products use the SELL-32-512 layout built in
// dec_sell.cu: one warp per slice of 32 rows, one lane per row.
//
//   FP64 mode : x, r, z, p, q in FP64; L and the preconditioner in FP64.
//   mixed mode: PCG with FP32 vectors and L and a BF16 FSAI factor (or an
//               FP32 Jacobi), whose residual is replaced by the FP64 residual
//               b - L x of an FP64 solution x every time it has dropped by
//               1e-2 (defect correction that keeps the search direction).
#include "dec_kern.cuh"

#include <algorithm>
#include <cmath>

namespace dec {

// ------------------------------------------------------------ kernels
// Element-wise kernels run grid_vec blocks (grid-stride over rows); SELL
// kernels run grid_sell blocks, one slice per warp.

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

// Scalars of an FP64 CG that starts from x0 != 0 (a warm start): the
// residual r = b - L x0 and its r.r (*rr_in) are already computed; here
// |b|^2 (the stopping rule stays ||b - L x|| <= rtol ||b||), p = 0.
__global__ void __launch_bounds__(kBlock)
cg_warm_init_kernel(int64_t n, const double* __restrict__ b, double* __restrict__ p,
                    double rtol2, const double* __restrict__ rr_in, CgScalars* cg,
                    double* partial, unsigned* ticket) {
  double bb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    bb += b[i] * b[i];
    p[i] = 0.0;
  }
  double v[1] = {bb}, t[1];
  if (grid_reduce<kBlock, 1>(v, t, partial, ticket) && threadIdx.x == 0) {
    const double rr = *rr_in;
    cg->bnorm2 = t[0];
    cg->tol2 = rtol2 * t[0];
    cg->rr = rr;
    cg->done = (t[0] == 0.0 || rr <= rtol2 * t[0]) ? 1 : 0;
    cg->iters = 0;
    cg->breakdown = 0;
    cg->beta = 0.0;
    cg->rz = 0.0;
  }
}

// *out = |b|^2
__global__ void __launch_bounds__(kBlock)
sq_norm_kernel(int64_t n, const double* __restrict__ b, double* out, double* partial,
               unsigned* ticket) {
  double bb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    bb += b[i] * b[i];
  double v[1] = {bb}, t[1];
  if (grid_reduce<kBlock, 1>(v, t, partial, ticket) && threadIdx.x == 0) *out = t[0];
}

// Widths (entries per row) staged in shared memory by the SELL kernels.
// The FSAI halves (at most 14 entries per row on the Delaunay meshes here)
// are staged: their BF16 apply ran 1.3-1.5x faster than with register
// chunks.  L (16 per row on average, 26 at most) keeps register chunks
// (kStageL = 0): staging its wider slices cut the resident warps and ran
// slower, in FP64 and in FP32.
#ifndef DEC_STAGE_L
#define DEC_STAGE_L 0
#endif
#ifndef DEC_STAGE_G
#define DEC_STAGE_G 14
#endif
// entries per register chunk of L's row product (unstaged)
#ifndef DEC_CHUNK_L
#define DEC_CHUNK_L 8
#endif
// resident blocks per SM the unstaged SELL kernels are sized for
#ifndef DEC_SELL_PER_SM
#define DEC_SELL_PER_SM 4
#endif
constexpr int kStageL = DEC_STAGE_L;
constexpr int kStageG = DEC_STAGE_G;
constexpr int kChunkL = DEC_CHUNK_L;
// The mixed mode runs as one persistent kernel up to this many nodes (its
// 3 grid barriers per iteration beat 5 launches when the matrices sit in
// L2) and as per-phase kernels above (more warps in flight per SM: 1.5x
// faster per iteration at 128^3).
constexpr int64_t kPersistMaxRows = 400000;

// Dynamic shared memory of a SELL kernel block and the number of its blocks:
// one slice per warp, at most 4 resident blocks per SM (the reduction
// partials are sized for 4 * SMs blocks), fewer when the stage is large.
template <int WMAX, typename MT>
constexpr int sell_smem() {
  return WMAX ? (kBlock / 32) * stage_bytes<WMAX, MT>() : 0;
}
template <int WMAX, typename MT>
static unsigned sell_grid(const dec_ctx* ctx, int64_t nslices) {
  constexpr int smem = sell_smem<WMAX, MT>();
  const int per_sm = smem ? std::max(1, std::min(4, (200 * 1024) / smem)) : DEC_SELL_PER_SM;
  return (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((nslices + kBlock / 32 - 1) / (kBlock / 32),
                           (int64_t)ctx->num_sms * per_sm));
}

// the warp's shared-memory stage (WMAX > 0) or nullptr
template <int WMAX, typename MT>
__device__ __forceinline__ unsigned char* warp_stage() {
  extern __shared__ __align__(16) unsigned char dsm[];
  if constexpr (WMAX > 0) return dsm + (threadIdx.x >> 5) * stage_bytes<WMAX, MT>();
  else return nullptr;
}

// body(row, (A x)_row) over every row, one slice per warp at a time
template <int WMAX, int CHUNK, typename MT, typename VT, typename Body>
__device__ __forceinline__ void for_rows(const SellArg<MT>& A, const VT* __restrict__ x,
                                         Body&& body) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (kBlock / 32);
  const int64_t first = blockIdx.x * (int64_t)(kBlock / 32) + (threadIdx.x >> 5);
  unsigned char* st = warp_stage<WMAX, MT>();
  for (int64_t s = first; s < A.nslices; s += warps) {
    const int32_t r = __ldg(A.perm + 32 * s + lane);
    VT acc;
    if constexpr (WMAX > 0) acc = sell_row_staged<WMAX>(A, s, lane, x, st);
    else acc = sell_row<MT, VT, CHUNK>(A, s, lane, x);
    if (r >= 0) body(r, acc);
  }
}

// q = A p and alpha = (r.z) / (p.q); CHUNK entries per register round trip
template <int WMAX, int CHUNK, typename MT, typename VT>
__global__ void __launch_bounds__(kBlock)
spmv_pq_kernel(SellArg<MT> A, const VT* __restrict__ p, VT* __restrict__ q,
               CgScalars* cg, double* partial, unsigned* ticket) {
  if (*(volatile int*)&cg->done) return;
  double pq = 0.0;
  for_rows<WMAX, CHUNK>(A, p, [&](int32_t r, VT acc) {
    q[r] = acc;
    pq += to_d(p[r]) * to_d(acc);
  });
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

// x += alpha p, r -= alpha q, r.r; with Jacobi also z = dinv r and r.z.
// Element-wise kernels run few blocks with 4 elements per thread in flight:
// GB300's FP64 pipe is narrow, so the per-warp cost of the FP64 reductions
// has to be spread over several elements per thread.  Per-thread sums are
// kept in the vector type and widened to FP64 before the warp reduction.
template <typename VT, typename DT, bool JACOBI>
__global__ void __launch_bounds__(kBlock)
update_kernel(int64_t n, VT* __restrict__ x, VT* __restrict__ r,
              const VT* __restrict__ p, const VT* __restrict__ q,
              const DT* __restrict__ dinv, VT* __restrict__ z, int max_iter,
              CgScalars* cg, double* partial, unsigned* ticket) {
  if (*(volatile int*)&cg->done) return;
  const VT alpha = (VT)cg->alpha;
  VT rr = VT(0), rz = VT(0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  auto one = [&](int64_t k, VT pk, VT qk, VT xk, VT rk) {
    const VT ri = fma_(-alpha, qk, rk);
    x[k] = fma_(alpha, pk, xk);
    r[k] = ri;
    rr = fma_(ri, ri, rr);
    if (JACOBI) {
      const VT zi = (VT)dinv[k] * ri;
      z[k] = zi;
      rz = fma_(ri, zi, rz);
    }
  };
  for (; i + 3 * stride < n; i += 4 * stride) {
    VT pv[4], qv[4], xv[4], rv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = i + u * stride;
      pv[u] = p[k]; qv[u] = q[k]; xv[u] = x[k]; rv[u] = r[k];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) one(i + u * stride, pv[u], qv[u], xv[u], rv[u]);
  }
  for (; i < n; i += stride) one(i, p[i], q[i], x[i], r[i]);
  if (JACOBI) {
    double v[2] = {to_d(rr), to_d(rz)}, t[2];
    if (grid_reduce<kBlock, 2>(v, t, partial, ticket) && threadIdx.x == 0) {
      cg->rr = t[0];
      cg->iters += 1;
      if (t[0] <= cg->tol2 || cg->iters >= max_iter || !isfinite(t[0])) cg->done = 1;
      cg->beta = t[1] / cg->rz;
      cg->rz = t[1];
    }
  } else {
    double v[1] = {to_d(rr)}, t[1];
    if (grid_reduce<kBlock, 1>(v, t, partial, ticket) && threadIdx.x == 0) {
      cg->rr = t[0];
      cg->iters += 1;
      if (t[0] <= cg->tol2 || cg->iters >= max_iter || !isfinite(t[0])) cg->done = 1;
    }
  }
}

// y = A x (FSAI first half: t = G r)
template <int WMAX, typename MT, typename VT>
__global__ void __launch_bounds__(kBlock)
sell_apply_kernel(SellArg<MT> A, const VT* __restrict__ x, VT* __restrict__ y,
                  const CgScalars* cg) {
  if (*(volatile const int*)&cg->done) return;
  for_rows<WMAX, 8>(A, x, [&](int32_t r, VT acc) { y[r] = acc; });
}

// z = A t (FSAI second half: z = G^T t), r.z, then beta = (r.z)_new /
// (r.z)_old.  `init` keeps beta = 0.
template <int WMAX, typename MT, typename VT>
__global__ void __launch_bounds__(kBlock)
sell_apply_dot_kernel(SellArg<MT> A, const VT* __restrict__ t,
                      const VT* __restrict__ r, VT* __restrict__ z, int init,
                      CgScalars* cg, double* partial, unsigned* ticket) {
  if (*(volatile int*)&cg->done) return;
  double rz = 0.0;
  for_rows<WMAX, 8>(A, t, [&](int32_t row, VT acc) {
    z[row] = acc;
    rz += to_d(r[row]) * to_d(acc);
  });
  double v[1] = {rz}, tt[1];
  if (grid_reduce<kBlock, 1>(v, tt, partial, ticket) && threadIdx.x == 0) {
    cg->beta = init ? 0.0 : tt[0] / cg->rz;
    cg->rz = tt[0];
  }
}

// Jacobi at a (re)start: z = dinv r, r.z; `init` sets beta = 0, otherwise
// beta = (r.z)_new / (r.z)_old keeps the search direction
template <typename VT, typename DT>
__global__ void __launch_bounds__(kBlock)
jacobi_init_kernel(int64_t n, const DT* __restrict__ dinv, const VT* __restrict__ r,
                   VT* __restrict__ z, int init, CgScalars* cg, double* partial,
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
    cg->beta = init ? 0.0 : t[0] / cg->rz;
    cg->rz = t[0];
  }
}

// Start a new segment of the FP32 iteration after a reliable update: stop
// again once r.r has dropped by `delta2` from the new (FP64) residual.
__global__ void segment_kernel(CgScalars* cg, const double* rr64, double delta2,
                               int restart) {
  cg->tol2 = delta2 * *rr64;
  cg->rr = *rr64;
  cg->done = 0;
  if (restart) cg->breakdown = 0;
}

// p = z + beta p
template <typename VT>
__global__ void __launch_bounds__(kBlock)
xpay_kernel(int64_t n, const VT* __restrict__ z, VT* __restrict__ p,
            const CgScalars* cg) {
  if (*(volatile const int*)&cg->done) return;
  const VT beta = (VT)cg->beta;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {
    VT zv[4], pv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) { zv[u] = z[i + u * stride]; pv[u] = p[i + u * stride]; }
#pragma unroll
    for (int u = 0; u < 4; ++u) p[i + u * stride] = fma_(beta, pv[u], zv[u]);
  }
  for (; i < n; i += stride) p[i] = fma_(beta, p[i], z[i]);
}

// FP64 residual r = b - A x, r.r into *out; optionally r32 = (float) r
__global__ void __launch_bounds__(kBlock)
residual_kernel(SellArg<double> A, const double* __restrict__ x,
                const double* __restrict__ b, double* __restrict__ r,
                float* __restrict__ r32, double* out, double* partial,
                unsigned* ticket) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (kBlock / 32);
  double rr = 0.0;
  for (int64_t s = blockIdx.x * (int64_t)(kBlock / 32) + (threadIdx.x >> 5);
       s < A.nslices; s += warps) {
    const int32_t row = __ldg(A.perm + 32 * s + lane);
    const double acc = sell_row(A, s, lane, x);
    if (row >= 0) {
      const double ri = b[row] - acc;
      r[row] = ri;
      if (r32) r32[row] = (float)ri;
      rr += ri * ri;
    }
  }
  double v[1] = {rr}, t[1];
  if (grid_reduce<kBlock, 1>(v, t, partial, ticket) && threadIdx.x == 0) *out = t[0];
}

// x64 += e32, e32 = 0
__global__ void __launch_bounds__(kBlock)
correct_kernel(int64_t n, double* __restrict__ x, float* __restrict__ e) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += (double)e[i];
    e[i] = 0.0f;
  }
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

// Opt every staged SELL kernel into its dynamic shared memory (the FP64
// stage of L is above the 48 KB default).
cudaError_t init_kernel_attributes() {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f, int bytes) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  };
  set((const void*)spmv_pq_kernel<kStageL, kChunkL, double, double>,
      sell_smem<kStageL, double>());
  set((const void*)spmv_pq_kernel<kStageL, kChunkL, float, float>, sell_smem<kStageL, float>());
  set((const void*)sell_apply_kernel<kStageG, double, double>, sell_smem<kStageG, double>());
  set((const void*)sell_apply_dot_kernel<kStageG, double, double>, sell_smem<kStageG, double>());
  set((const void*)sell_apply_kernel<kStageG, __nv_bfloat16, float>,
      sell_smem<kStageG, __nv_bfloat16>());
  set((const void*)sell_apply_dot_kernel<kStageG, __nv_bfloat16, float>,
      sell_smem<kStageG, __nv_bfloat16>());
  return e;
}

// k_eff pieces of every instance: block row blockIdx.y takes instances
// kKeffGroup * y ... (crack state b when `states`, Dirichlet set b when
// `sets`, field b when `fields`), reading each row's structure and edge data
// once for the whole group; T = u_b + T0 on Dirichlet nodes is formed on the
// fly.  Block partials go to partial[(3 b + v) * gridDim.x + block] and
// k_eff_batch_sum_kernel adds them in block order (deterministic).
constexpr int kKeffGroup = 8;

__global__ void __launch_bounds__(kBlock)
k_eff_batch_kernel(int64_t n, int B, const int32_t* __restrict__ rowptr,
                   const int32_t* __restrict__ col, const int32_t* __restrict__ eid,
                   const int32_t* __restrict__ dpos, const uint8_t* __restrict__ tag,
                   const double* __restrict__ xyz, const double* __restrict__ w0,
                   int64_t ne, const uint8_t* __restrict__ fc, int states, int sets,
                   int fields, const double* __restrict__ u, const double* __restrict__ T0,
                   double* __restrict__ partial) {
  __shared__ double sh[kBlock];
  const int g0 = blockIdx.y * kKeffGroup;
  const int gn = min(kKeffGroup, B - g0);
  auto Tof = [&](int b, int64_t i) {
    const double* t0 = T0 + (sets ? (int64_t)b * n : 0);
    return u[(int64_t)b * n + i] + (tag[i] == DEC_NODE_DIRICHLET ? t0[i] : 0.0);
  };
  double qin[kKeffGroup], qout[kKeffGroup], en[kKeffGroup];
#pragma unroll
  for (int j = 0; j < kKeffGroup; ++j) qin[j] = qout[j] = en[j] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double Ti[kKeffGroup], net[kKeffGroup];
#pragma unroll
    for (int j = 0; j < kKeffGroup; ++j) {
      Ti[j] = j < gn ? Tof(g0 + j, i) : 0.0;
      net[j] = 0.0;
    }
    const int32_t k0 = rowptr[i], k1 = rowptr[i + 1], kd = dpos[i];
    for (int32_t k = k0; k < k1; ++k) {
      if (k == kd) continue;
      const int32_t e = eid[k];
      const int32_t c = col[k];
      const int f = (int)fc[e];
      const double ws = fields ? 0.0 : w0[e];
#pragma unroll
      for (int j = 0; j < kKeffGroup; ++j) {
        if (j >= gn) break;
        const int b = g0 + j;
        const double wb = fields ? w0[(int64_t)b * ne + e] : ws;
        const double we = f > (states ? b : 0) ? wb : 0.0;
        const double d = Ti[j] - Tof(b, c);
        net[j] += we * d;
        if (k > kd) en[j] += we * d * d;
      }
    }
    if (tag[i] == DEC_NODE_DIRICHLET) {
      const double xi = xyz[3 * i];
#pragma unroll
      for (int j = 0; j < kKeffGroup; ++j) {
        if (xi == 0.0) qin[j] += net[j];
        else if (xi == 1.0) qout[j] -= net[j];
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kKeffGroup; ++j) {
    const double v[3] = {qin[j], qout[j], en[j]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double t = block_sum<kBlock>(v[k], sh);
      if (threadIdx.x == 0 && j < gn)
        partial[(3 * (int64_t)(g0 + j) + k) * gridDim.x + blockIdx.x] = t;
    }
  }
}

// one warp per value: lane l adds partials l, l + 32, ... and the warp sum
// combines the lanes in a fixed order
__global__ void k_eff_batch_sum_kernel(int nblocks, int nvals, const double* __restrict__ partial,
                                       double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < nvals;
       v += (gridDim.x * blockDim.x) >> 5) {
    double s = 0.0;
    for (int k = lane; k < nblocks; k += 32) s += partial[(int64_t)v * nblocks + k];
    s = warp_sum(s);
    if (lane == 0) out[v] = s;
  }
}

dec_status k_eff_all(dec_ctx* ctx, double* out3_host) {
  const int64_t n = ctx->n;
  const int B = ctx->B;
  cudaStream_t s = ctx->stream;
  const unsigned G = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((n + kBlock - 1) / kBlock, (int64_t)ctx->num_sms * 4));
  const unsigned GY = (unsigned)((B + kKeffGroup - 1) / kKeffGroup);
  DEC_TRY(ctx->kpartial.ensure((size_t)3 * B * G));
  DEC_TRY(ctx->out3.ensure(3 * (size_t)B + 2));
  k_eff_batch_kernel<<<dim3(G, GY), kBlock, 0, s>>>(
      n, B, ctx->rowptr.p, ctx->col.p, ctx->eid.p, ctx->dpos.p, ctx->tag.p, ctx->xyz.p, ctx->w.p,
      ctx->ne, ctx->first_cut.p, ctx->n_scales > 1, ctx->n_sets > 1, ctx->n_fields > 1,
      ctx->u.p, ctx->T0.p, ctx->kpartial.p);
  k_eff_batch_sum_kernel<<<(unsigned)((3 * B + 3) / 4), 128, 0, s>>>(
      (int)G, 3 * B, ctx->kpartial.p, ctx->out3.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 2;
  DEC_TRY(cudaMemcpyAsync(out3_host, ctx->out3.p, 3 * sizeof(double) * B,
                          cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaStreamSynchronize(s));
  return DEC_OK;
}

// ------------------------------------------------------- launch shapes
// The single-instance SELL kernels run in one of a few launch shapes,
// picked at run time per problem size (nodes, matrix entries) and
// precision by sell_tune: for L, register round trips of 4, 8 or 12
// entries at 4 or 8 resident blocks per SM (code 100 * blocks + entries);
// for the FSAI halves, staged slices (code 14) or register round trips of 8
// (code 8).  Every shape adds a row's entries in the same order, so the
// choice never changes a result.
struct LShape {
  int chunk, per_sm;
};
constexpr int kNumLShapes = 4;
constexpr LShape kLShapes[kNumLShapes] = {{8, 4}, {8, 8}, {12, 4}, {4, 8}};
constexpr int kNumGShapes = 2;
constexpr int kGShapeCode[kNumGShapes] = {kStageG, 8};

static int lshape_code(int v) { return 100 * kLShapes[v].per_sm + kLShapes[v].chunk; }

static unsigned sell_grid_n(const dec_ctx* ctx, int64_t nslices, int per_sm) {
  return (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((nslices + kBlock / 32 - 1) / (kBlock / 32),
                           (int64_t)ctx->num_sms * per_sm));
}

template <typename MT, typename VT>
static void launch_spmv_pq(dec_ctx* ctx, int v, const SellArg<MT>& A, const VT* p, VT* q,
                           CgScalars* cg, double* part, unsigned* tk) {
  static_assert(kStageL == 0, "L shapes are register round trips");
  const unsigned g = sell_grid_n(ctx, A.nslices, kLShapes[v].per_sm);
  cudaStream_t s = ctx->stream;
  switch (kLShapes[v].chunk) {
    case 4: spmv_pq_kernel<0, 4, MT, VT><<<g, kBlock, 0, s>>>(A, p, q, cg, part, tk); break;
    case 12: spmv_pq_kernel<0, 12, MT, VT><<<g, kBlock, 0, s>>>(A, p, q, cg, part, tk); break;
    default: spmv_pq_kernel<0, 8, MT, VT><<<g, kBlock, 0, s>>>(A, p, q, cg, part, tk); break;
  }
}

// t = G r, then z = G^T t with r.z (beta as sell_apply_dot_kernel)
template <typename PT, typename VT>
static void launch_fsai(dec_ctx* ctx, int v, const SellArg<PT>& Glo, const SellArg<PT>& Gup,
                        const VT* r, VT* t, VT* z, int init, CgScalars* cg, double* part,
                        unsigned* tk) {
  cudaStream_t s = ctx->stream;
  if (v == 0) {
    constexpr int SG = sell_smem<kStageG, PT>();
    sell_apply_kernel<kStageG, PT, VT><<<sell_grid<kStageG, PT>(ctx, Glo.nslices), kBlock, SG,
                                         s>>>(Glo, r, t, cg);
    sell_apply_dot_kernel<kStageG, PT, VT><<<sell_grid<kStageG, PT>(ctx, Gup.nslices), kBlock,
                                             SG, s>>>(Gup, t, r, z, init, cg, part, tk);
  } else {
    sell_apply_kernel<0, PT, VT><<<sell_grid_n(ctx, Glo.nslices, 4), kBlock, 0, s>>>(Glo, r, t,
                                                                                    cg);
    sell_apply_dot_kernel<0, PT, VT><<<sell_grid_n(ctx, Gup.nslices, 4), kBlock, 0, s>>>(
        Gup, t, r, z, init, cg, part, tk);
  }
}

// Autotuner of the shapes above: the first phased solve of a problem size in
// a precision (0: FP64, 1: FP32 / BF16) times 3 launches of each shape
// (after one untimed) on the context's scratch vectors and keeps the
// fastest; a shape set by dec_set_sell_variant is used instead.
template <typename MT, typename PT, typename VT>
static dec_status sell_tune(dec_ctx* ctx, int prec, const SellArg<MT>& A,
                            const SellArg<PT>& Glo, const SellArg<PT>& Gup, bool fsai,
                            VT* v0, VT* v1, VT* v2) {
  if (ctx->sell_force_l >= 0) ctx->sell_l[prec] = ctx->sell_force_l;
  if (ctx->sell_force_g >= 0) ctx->sell_g[prec] = ctx->sell_force_g;
  const bool same = ctx->sell_key[prec][0] == ctx->n && ctx->sell_key[prec][1] == ctx->nnz;
  const bool need_l = ctx->sell_force_l < 0 && (!same || ctx->sell_l[prec] < 0);
  const bool need_g = fsai && ctx->sell_force_g < 0 && (!same || ctx->sell_g[prec] < 0);
  if (!need_l && !need_g) return DEC_OK;
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n;
  DEC_TRY(cudaMemsetAsync(v0, 0, sizeof(VT) * n, s));
  CgScalars h{};
  h.rz = 1.0;
  cudaEvent_t e0, e1;
  DEC_TRY(cudaEventCreate(&e0));
  DEC_TRY(cudaEventCreate(&e1));
  auto timed = [&](auto&& launch, float* ms) -> dec_status {
    float tot = 0.0f;
    for (int rep = 0; rep < 4; ++rep) {
      DEC_TRY(cudaMemcpyAsync(ctx->cg.p, &h, sizeof(h), cudaMemcpyHostToDevice, s));
      DEC_TRY(cudaEventRecord(e0, s));
      launch();
      DEC_TRY(cudaEventRecord(e1, s));
      DEC_TRY(cudaEventSynchronize(e1));
      float m = 0.0f;
      DEC_TRY(cudaEventElapsedTime(&m, e0, e1));
      if (rep > 0) tot += m;
    }
    *ms = tot;
    return DEC_OK;
  };
  dec_status st = DEC_OK;
  if (need_l) {
    float best = 0.0f;
    for (int v = 0; v < kNumLShapes && st == DEC_OK; ++v) {
      float ms = 0.0f;
      st = timed([&] { launch_spmv_pq<MT, VT>(ctx, v, A, v0, v1, ctx->cg.p, ctx->partial.p,
                                             ctx->ticket.p); }, &ms);
      ctx->launches += 4;
      if (v == 0 || ms < best) { best = ms; ctx->sell_l[prec] = v; }
    }
  }
  if (need_g && st == DEC_OK) {
    float best = 0.0f;
    for (int v = 0; v < kNumGShapes && st == DEC_OK; ++v) {
      float ms = 0.0f;
      st = timed([&] { launch_fsai<PT, VT>(ctx, v, Glo, Gup, v0, v1, v2, 1, ctx->cg.p,
                                           ctx->partial.p, ctx->ticket.p); }, &ms);
      ctx->launches += 8;
      if (v == 0 || ms < best) { best = ms; ctx->sell_g[prec] = v; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DEC_OK) return st;
  DEC_TRY(cudaGetLastError());
  ctx->sell_key[prec][0] = ctx->n;
  ctx->sell_key[prec][1] = ctx->nnz;
  return DEC_OK;
}

// ------------------------------------------------------------- driver
constexpr int kChunk = 16;       // iterations per graph launch / host poll

// Operators of one precision: L, the two FSAI halves (or Jacobi).
template <typename MT, typename PT, typename DT>
struct Ops {
  SellArg<MT> A;
  SellArg<PT> Glo, Gup;
  const DT* dinv;
};

template <typename VT, typename MT, typename PT, typename DT>
static void launch_iterations(dec_ctx* ctx, int64_t n, const Ops<MT, PT, DT>& op,
                              VT* x, VT* r, VT* z, VT* p, VT* q, VT* t, int max_iter,
                              int count) {
  cudaStream_t s = ctx->stream;
  const unsigned G = (unsigned)ctx->grid_vec;
  const int prec = sizeof(VT) == sizeof(double) ? 0 : 1;
  const int vl = std::max(ctx->sell_l[prec], 0), vg = std::max(ctx->sell_g[prec], 0);
  CgScalars* cg = ctx->cg.p;
  double* part = ctx->partial.p;
  unsigned* tk = ctx->ticket.p;
  const bool jac = ctx->precond == DEC_PRECOND_JACOBI;
  ctx->launches += (int64_t)count * (jac ? 3 : 5);
  for (int it = 0; it < count; ++it) {
    launch_spmv_pq<MT, VT>(ctx, vl, op.A, p, q, cg, part, tk);
    if (jac) {
      update_kernel<VT, DT, true><<<G, kBlock, 0, s>>>(n, x, r, p, q, op.dinv, z,
                                                       max_iter, cg, part, tk);
    } else {
      update_kernel<VT, DT, false><<<G, kBlock, 0, s>>>(n, x, r, p, q, op.dinv, z,
                                                        max_iter, cg, part, tk);
      launch_fsai<PT, VT>(ctx, vg, op.Glo, op.Gup, r, t, z, 0, cg, part, tk);
    }
    xpay_kernel<VT><<<G, kBlock, 0, s>>>(n, z, p, cg);
  }
}

// (Re)start from the current r: z = M r, r.z and p = z (init) or, after a
// reliable update that keeps the search direction, p = z + beta p with
// beta = (r.z)_new / (r.z)_old.
template <typename VT, typename MT, typename PT, typename DT>
static void launch_restart(dec_ctx* ctx, int64_t n, const Ops<MT, PT, DT>& op, VT* r,
                           VT* z, VT* p, VT* t, int init = 1) {
  cudaStream_t s = ctx->stream;
  const unsigned G = (unsigned)ctx->grid_vec;
  const int prec = sizeof(VT) == sizeof(double) ? 0 : 1;
  CgScalars* cg = ctx->cg.p;
  ctx->launches += ctx->precond == DEC_PRECOND_JACOBI ? 2 : 3;
  if (ctx->precond == DEC_PRECOND_JACOBI) {
    jacobi_init_kernel<VT, DT><<<G, kBlock, 0, s>>>(n, op.dinv, r, z, init, cg,
                                                    ctx->partial.p, ctx->ticket.p);
  } else {
    launch_fsai<PT, VT>(ctx, std::max(ctx->sell_g[prec], 0), op.Glo, op.Gup, r, t, z, init,
                        cg, ctx->partial.p, ctx->ticket.p);
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
static dec_status run_pcg(dec_ctx* ctx, int64_t n, const Ops<MT, PT, DT>& op, VT* x,
                          VT* r, VT* z, VT* p, VT* q, VT* t, int max_iter,
                          CgScalars* h) {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const int64_t per_chunk = (int64_t)kChunk * (ctx->precond == DEC_PRECOND_JACOBI ? 3 : 5);
  DEC_TRY(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  launch_iterations<VT, MT, PT, DT>(ctx, n, op, x, r, z, p, q, t, max_iter, kChunk);
  ctx->launches -= per_chunk;  // counted per replay below
  cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
  if (ce != cudaSuccess) return ctx->cuda_fail(ce, "cudaStreamEndCapture");
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return ctx->cuda_fail(ce, "cudaGraphInstantiate");
  dec_status st = DEC_OK;
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
                          int mode, int* iters_out, double* relres_out, bool warm) {
  const int64_t n = ctx->n;
  const int vs = value_set(ctx, inst);
  cudaStream_t s = ctx->stream;
  const unsigned G = (unsigned)ctx->grid_vec, Gs = (unsigned)ctx->grid_sell;
  const SellArg<double> A64 = sell_arg(ctx->sellL, ctx->sL64.p + (int64_t)vs * ctx->sellL.total);
  const double* bvec = ctx->b.p + (int64_t)inst * n;
  double* u = ctx->u.p + (int64_t)inst * n;
  CgScalars h{};
  double* rr_dev = ctx->out3.p + 3 * (int64_t)ctx->B;  // scratch scalar
  double rr_true = 0.0, bnorm2 = 0.0;
  int total_iters = 0;
  dec_status st = DEC_OK;
  const bool fsai = ctx->precond == DEC_PRECOND_FSAI;

  if (mode == DEC_MODE_FP64) {
    Ops<double, double, double> op{
        A64,
        sell_arg(ctx->sellLo, fsai ? ctx->sGlo64.p + (int64_t)vs * ctx->sellLo.total : nullptr),
        sell_arg(ctx->sellUp, fsai ? ctx->sGup64.p + (int64_t)vs * ctx->sellUp.total : nullptr),
        fsai ? nullptr : ctx->dinv64.p + (int64_t)vs * n};
    double *x = ctx->x64.p, *r = ctx->r64.p, *z = ctx->z64.p, *p = ctx->p64.p,
           *q = ctx->q64.p, *t = ctx->t64.p;
    DEC_TRY_STATUS(sell_tune(ctx, 0, op.A, op.Glo, op.Gup, fsai, t, q, z));
    if (warm) {
      // start from the current solution u: r = b - L u
      DEC_TRY(cudaMemcpyAsync(x, u, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      ctx->launches += 2;
      residual_kernel<<<Gs, kBlock, 0, s>>>(A64, x, bvec, r, nullptr, rr_dev, ctx->partial.p,
                                           ctx->ticket.p);
      cg_warm_init_kernel<<<G, kBlock, 0, s>>>(n, bvec, p, rtol * rtol, rr_dev, ctx->cg.p,
                                               ctx->partial.p, ctx->ticket.p);
    } else {
      ctx->launches += 1;
      cg_init_kernel<double, double><<<G, kBlock, 0, s>>>(n, bvec, x, r, p, rtol * rtol,
                                                          ctx->cg.p, ctx->partial.p,
                                                          ctx->ticket.p);
    }
    launch_restart<double>(ctx, n, op, r, z, p, t);
    DEC_TRY(cudaGetLastError());
    for (;;) {
      st = run_pcg<double>(ctx, n, op, x, r, z, p, q, t, max_iter, &h);
      if (st != DEC_OK) return st;
      bnorm2 = h.bnorm2;
      total_iters = h.iters;
      if (bnorm2 == 0.0) { rr_true = 0.0; break; }
      // true residual, replacing the recursive one
      ctx->launches += 1;
      residual_kernel<<<Gs, kBlock, 0, s>>>(A64, x, bvec, r, nullptr, rr_dev, ctx->partial.p,
                                           ctx->ticket.p);
      DEC_TRY(cudaMemcpyAsync(&rr_true, rr_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
      DEC_TRY(cudaStreamSynchronize(s));
      if (h.breakdown) { st = ctx->fail(DEC_ERR_BREAKDOWN, "CG breakdown: p.Lp <= 0 or not finite"); break; }
      if (rr_true <= rtol * rtol * bnorm2) break;
      if (h.iters >= max_iter) { st = ctx->fail(DEC_NOT_CONVERGED, "max_iter reached"); break; }
      // restart from the true residual
      int zero = 0;
      DEC_TRY(cudaMemcpyAsync(&ctx->cg.p->done, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
      launch_restart<double>(ctx, n, op, r, z, p, t);
      DEC_TRY(cudaGetLastError());
    }
    DEC_TRY(cudaMemcpyAsync(u, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  } else if (mode == DEC_MODE_MIXED && !warm && n <= kPersistMaxRows &&
             (st = solve_mixed_persistent(ctx, inst, rtol, max_iter, iters_out, relres_out)) !=
                 DEC_ERR_LIMIT) {
    return st;   // the whole mixed solve ran as one cooperative kernel
  } else {
    st = DEC_OK;
    // Mixed: one FP32 PCG whose residual is replaced, every time it has
    // dropped by kSegment since the last replacement, by the FP64 residual
    // b - L x of the FP64 solution x += (FP32 accumulated update) ("reliable
    // updates": defect correction that keeps the search direction, so the
    // iteration count stays close to FP64 CG).  Convergence is decided on
    // the FP64 residual only.
    Ops<float, __nv_bfloat16, float> op{
        sell_arg(ctx->sellL, ctx->sL32.p + (int64_t)vs * ctx->sellL.total),
        sell_arg(ctx->sellLo, fsai ? ctx->sGlo16.p + (int64_t)vs * ctx->sellLo.total : nullptr),
        sell_arg(ctx->sellUp, fsai ? ctx->sGup16.p + (int64_t)vs * ctx->sellUp.total : nullptr),
        fsai ? nullptr : ctx->dinv32.p + (int64_t)vs * n};
    constexpr double kSegment = 1e-4;   // r.r drop between replacements (1e-2 in norm)
    double* x64 = ctx->x64.p;
    double* r64 = ctx->r64.p;
    float *x = ctx->x32.p, *r = ctx->r32.p, *z = ctx->z32.p, *p = ctx->p32.p,
          *q = ctx->q32.p, *t = ctx->t32.p;
    DEC_TRY_STATUS(sell_tune(ctx, 1, op.A, op.Glo, op.Gup, fsai, t, q, z));
    // x64 = 0 (or the current solution u for a warm start)
    if (warm) DEC_TRY(cudaMemcpyAsync(x64, u, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    else DEC_TRY(cudaMemsetAsync(x64, 0, sizeof(double) * n, s));
    // r64 = b - L x64, r32 = (float) r64, |r|^2; the FP32 state starts from r32
    ctx->launches += 2;
    residual_kernel<<<Gs, kBlock, 0, s>>>(A64, x64, bvec, r64, q, rr_dev, ctx->partial.p,
                                         ctx->ticket.p);
    cg_init_kernel<float, float><<<G, kBlock, 0, s>>>(n, q, x, r, p, kSegment, ctx->cg.p,
                                                      ctx->partial.p, ctx->ticket.p);
    DEC_TRY(cudaMemcpyAsync(&rr_true, rr_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (warm) {
      ctx->launches += 1;
      sq_norm_kernel<<<G, kBlock, 0, s>>>(n, bvec, rr_dev + 1, ctx->partial.p, ctx->ticket.p);
      DEC_TRY(cudaMemcpyAsync(&bnorm2, rr_dev + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    launch_restart<float>(ctx, n, op, r, z, p, t, 1);
    DEC_TRY(cudaGetLastError());
    DEC_TRY(cudaStreamSynchronize(s));
    if (!warm) bnorm2 = rr_true;
    double best = rr_true;
    int stall = 0;
    while (bnorm2 > 0.0 && rr_true > rtol * rtol * bnorm2) {
      st = run_pcg<float>(ctx, n, op, x, r, z, p, q, t, max_iter, &h);
      if (st != DEC_OK) return st;
      total_iters = h.iters;
      // reliable update: x64 += x32, x32 = 0, r64 = b - L x64, r32 = (float) r64
      ctx->launches += 2;
      correct_kernel<<<G, kBlock, 0, s>>>(n, x64, x);
      residual_kernel<<<Gs, kBlock, 0, s>>>(A64, x64, bvec, r64, r, rr_dev, ctx->partial.p,
                                           ctx->ticket.p);
      DEC_TRY(cudaMemcpyAsync(&rr_true, rr_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
      DEC_TRY(cudaStreamSynchronize(s));
      if (rr_true <= rtol * rtol * bnorm2) break;
      if (h.iters >= max_iter) { st = ctx->fail(DEC_NOT_CONVERGED, "max_iter reached"); break; }
      if (rr_true < 0.5 * best) { best = rr_true; stall = 0; }
      else if (++stall >= 4) { st = ctx->fail(DEC_NOT_CONVERGED, "residual replacement stalled"); break; }
      // next segment; after a breakdown or a stall restart the direction too
      const int restart = (h.breakdown || stall > 0) ? 1 : 0;
      ctx->launches += 1;
      segment_kernel<<<1, 1, 0, s>>>(ctx->cg.p, rr_dev, kSegment, restart);
      launch_restart<float>(ctx, n, op, r, z, p, t, restart);
      DEC_TRY(cudaGetLastError());
    }
    DEC_TRY(cudaMemcpyAsync(u, x64, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  *iters_out = total_iters;
  *relres_out = bnorm2 > 0.0 ? std::sqrt(rr_true / bnorm2) : 0.0;
  return st;
}

dec_status form_T(dec_ctx* ctx, int inst, double* T) {
  const int ts = ctx->n_sets > 1 ? inst : 0;
  ctx->launches += 1;
  form_T_kernel<<<(unsigned)ctx->grid_vec, kBlock, 0, ctx->stream>>>(
      ctx->n, ctx->u.p + (int64_t)inst * ctx->n, ctx->T0.p + (int64_t)ts * ctx->n,
      ctx->tag.p, T);
  DEC_TRY(cudaGetLastError());
  return DEC_OK;
}

// Time `reps` launches of one solver kernel on instance 0's data, each
// preceded (outside the timed events) by a write of `flush_bytes` to evict
// L2, so the figure is the cold-cache duration of a launch.
dec_status time_kernel(dec_ctx* ctx, int which, int reps, size_t flush_bytes,
                       double* avg_ms) {
  const int64_t n = ctx->n;
  cudaStream_t s = ctx->stream;
  DEC_TRY(ctx->flush.ensure(flush_bytes > 0 ? flush_bytes : 1));
  for (auto* bf : {&ctx->p64, &ctx->q64, &ctx->t64, &ctx->z64, &ctx->r64}) DEC_TRY(bf->ensure(n));
  for (auto* bf : {&ctx->p32, &ctx->q32, &ctx->t32, &ctx->z32, &ctx->r32}) DEC_TRY(bf->ensure(n));
  // finite operands: p = r = b (FP64), zeros (FP32), done = 0
  DEC_TRY(cudaMemcpyAsync(ctx->p64.p, ctx->b.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  DEC_TRY(cudaMemcpyAsync(ctx->r64.p, ctx->b.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  DEC_TRY(cudaMemsetAsync(ctx->p32.p, 0, sizeof(float) * n, s));
  DEC_TRY(cudaMemsetAsync(ctx->r32.p, 0, sizeof(float) * n, s));
  CgScalars h{};
  h.rz = 1.0;
  DEC_TRY(cudaMemcpyAsync(ctx->cg.p, &h, sizeof(h), cudaMemcpyHostToDevice, s));
  const auto L64 = sell_arg(ctx->sellL, ctx->sL64.p);
  const auto L32 = sell_arg(ctx->sellL, ctx->sL32.p);
  const auto Glo64 = sell_arg(ctx->sellLo, ctx->sGlo64.p);
  const auto Gup64 = sell_arg(ctx->sellUp, ctx->sGup64.p);
  const auto Glo16 = sell_arg(ctx->sellLo, ctx->sGlo16.p);
  const auto Gup16 = sell_arg(ctx->sellUp, ctx->sGup16.p);
  cudaEvent_t e0, e1;
  DEC_TRY(cudaEventCreate(&e0));
  DEC_TRY(cudaEventCreate(&e1));
  double total = 0.0;
  dec_status st = DEC_OK;
  for (int it = 0; it < reps && st == DEC_OK; ++it) {
    if (flush_bytes) DEC_TRY(cudaMemsetAsync(ctx->flush.p, it & 0xff, flush_bytes, s));
    DEC_TRY(cudaMemcpyAsync(&ctx->cg.p->done, &h.done, sizeof(int), cudaMemcpyHostToDevice, s));
    DEC_TRY(cudaEventRecord(e0, s));
    switch (which) {
      // the shapes the autotuner picked (the defaults before any solve)
      case DEC_KERNEL_SPMV_F64:
        launch_spmv_pq<double, double>(ctx, std::max(ctx->sell_l[0], 0), L64, ctx->p64.p,
                                       ctx->q64.p, ctx->cg.p, ctx->partial.p, ctx->ticket.p);
        break;
      case DEC_KERNEL_SPMV_F32:
        launch_spmv_pq<float, float>(ctx, std::max(ctx->sell_l[1], 0), L32, ctx->p32.p,
                                     ctx->q32.p, ctx->cg.p, ctx->partial.p, ctx->ticket.p);
        break;
      case DEC_KERNEL_FSAI_F64:
        launch_fsai<double, double>(ctx, std::max(ctx->sell_g[0], 0), Glo64, Gup64,
                                    ctx->r64.p, ctx->t64.p, ctx->z64.p, 1, ctx->cg.p,
                                    ctx->partial.p, ctx->ticket.p);
        break;
      case DEC_KERNEL_FSAI_BF16:
        launch_fsai<__nv_bfloat16, float>(ctx, std::max(ctx->sell_g[1], 0), Glo16, Gup16,
                                          ctx->r32.p, ctx->t32.p, ctx->z32.p, 1, ctx->cg.p,
                                          ctx->partial.p, ctx->ticket.p);
        break;
      default:
        st = ctx->fail(DEC_ERR_ARG, "time_kernel: unknown kernel id");
        continue;
    }
    ctx->launches += (which >= DEC_KERNEL_FSAI_F64) ? 2 : 1;
    DEC_TRY(cudaEventRecord(e1, s));
    DEC_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    DEC_TRY(cudaEventElapsedTime(&ms, e0, e1));
    total += ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == DEC_OK) *avg_ms = total / reps;
  return st;
}

}  // namespace dec

namespace dec {
int sell_l_code(int v) { return v < 0 ? 0 : lshape_code(v); }
int sell_g_code(int v) { return v < 0 ? 0 : kGShapeCode[v]; }
int sell_l_index(int code) {
  for (int v = 0; v < kNumLShapes; ++v)
    if (lshape_code(v) == code) return v;
  return -1;
}
int sell_g_index(int code) {
  for (int v = 0; v < kNumGShapes; ++v)
    if (kGShapeCode[v] == code) return v;
  return -1;
}
}  // namespace dec
