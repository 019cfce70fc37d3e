// dec_system.cu - values of the node Laplacian L = d0^T *1 d0 with the
// Dirichlet and zero-flux treatment of Sec. 2.3 (Eq. 11-13), the right-hand
// sides, and the preconditioners: Jacobi and a factored sparse approximate
// inverse (the ParaSails family of Sec. 2.3) on the pattern of lower(L).
#include "dec_internal.cuh"

#include <algorithm>

namespace dec {

// weight of edge e in crack state `state` (first_cut = first cut state)
__device__ __forceinline__ double edge_weight(const double* w, const uint8_t* fc,
                                              int32_t e, int state) {
  return (int)fc[e] > state ? w[e] : 0.0;
}

// Row i of L and b.  Off-diagonal -w_ij (0 towards Dirichlet nodes, whose
// values move to b), diagonal sum_j w_ij; Dirichlet rows and rows with all
// weights zero become identity rows with b = 0.
__device__ __forceinline__ void laplacian_row(
    int64_t i, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const int32_t* __restrict__ eid, const int32_t* __restrict__ dpos,
    const uint8_t* __restrict__ tag, const double* __restrict__ w,
    const uint8_t* __restrict__ fc, int state, const double* __restrict__ T0,
    double* __restrict__ val, double* __restrict__ b) {
  const int32_t k0 = rowptr[i], k1 = rowptr[i + 1], kd = dpos[i];
  if (tag[i] == DEC_NODE_DIRICHLET) {
    for (int32_t k = k0; k < k1; ++k) val[k] = k == kd ? 1.0 : 0.0;
    b[i] = 0.0;
    return;
  }
  double diag = 0.0, bi = 0.0;
  for (int32_t k = k0; k < k1; ++k) {
    if (k == kd) continue;
    const double we = edge_weight(w, fc, eid[k], state);
    diag += we;
    const int32_t j = col[k];
    double v;
    if (tag[j] == DEC_NODE_DIRICHLET) {
      v = 0.0;
      bi += we * T0[j];
    } else {
      v = we == 0.0 ? 0.0 : -we;
    }
    val[k] = v;
  }
  if (diag == 0.0) {  // isolated by cracks: decoupled identity row
    val[kd] = 1.0;
    b[i] = 0.0;
  } else {
    val[kd] = diag;
    b[i] = bi;
  }
}

// One thread per row.
__global__ void laplacian_values_kernel(
    int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const int32_t* __restrict__ eid, const int32_t* __restrict__ dpos,
    const uint8_t* __restrict__ tag, const double* __restrict__ w,
    const uint8_t* __restrict__ fc, int state, const double* __restrict__ T0,
    double* __restrict__ val, double* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    laplacian_row(i, rowptr, col, eid, dpos, tag, w, fc, state, T0, val, b);
}

__global__ void jacobi_kernel(int64_t n, const int32_t* __restrict__ dpos,
                              const double* __restrict__ val,
                              double* __restrict__ dinv64,
                              float* __restrict__ dinv32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double d = 1.0 / val[dpos[i]];
    dinv64[i] = d;
    if (dinv32) dinv32[i] = (float)d;
  }
}

// ------------------------------------------------------------------ FSAI
// One warp per row i.  P = columns of row i up to the diagonal (sorted,
// ending with i), k = |P| <= kFsaiMax.  The warp gathers A = L[P, P] into
// shared memory, factors A = C C^T (Cholesky, FP64) and back-substitutes
// C^T g = e_k: then g = A^-1 e_k * C_kk and g_k = 1 / C_kk, so g equals
// (A^-1 e_k) / sqrt((A^-1 e_k)_k), the FSAI row G[i, P].  A block whose
// Cholesky meets a pivot <= kPivotRel * max(diag A) is singular: it is
// factored again with kShiftRel * max(diag A) added to its diagonal.
constexpr int kFsaiMax = 32;
constexpr int kFsaiWarps = 4;
constexpr double kPivotRel = 1e-12;
constexpr double kShiftRel = 1e-12;

__device__ void fsai_gather(int lane, int k, const int32_t* P,
                            const int32_t* __restrict__ rowptr,
                            const int32_t* __restrict__ col,
                            const double* __restrict__ val, double (*A)[kFsaiMax + 1],
                            double shift) {
  for (int a = lane; a < k; a += 32) {
    for (int q = 0; q < k; ++q) A[a][q] = 0.0;
    const int32_t r = P[a];
    int q = 0;
    for (int32_t kk = rowptr[r]; kk < rowptr[r + 1] && q < k; ++kk) {
      const int32_t c = col[kk];
      while (q < k && P[q] < c) ++q;
      if (q < k && P[q] == c) A[a][q] = val[kk];
    }
    A[a][a] += shift;
  }
}

// returns false when a pivot is <= pivot_min (A is then partly overwritten)
__device__ bool fsai_cholesky(int lane, int k, double (*A)[kFsaiMax + 1],
                              double pivot_min) {
  for (int c = 0; c < k; ++c) {
    __syncwarp();
    const double d = A[c][c];
    if (!(d > pivot_min)) return false;
    const double lc = sqrt(d);
    __syncwarp();
    if (lane > c && lane < k) A[lane][c] /= lc;
    if (lane == c) A[c][c] = lc;
    __syncwarp();
    if (lane > c && lane < k) {
      const double lrc = A[lane][c];
      for (int q = c + 1; q <= lane; ++q) A[lane][q] -= lrc * A[q][c];
    }
  }
  __syncwarp();
  return true;
}

// Warp-per-row FSAI setup for the rows listed by the thread-per-row kernel
// (k > kFsaiThread); rows with k > kFsaiMax raise error bit 8.
__global__ void __launch_bounds__(32 * kFsaiWarps)
fsai_setup_list_kernel(const int32_t* __restrict__ rows, const int32_t* __restrict__ count,
                       const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                       const int32_t* __restrict__ eid, const int32_t* __restrict__ dpos,
                       const int32_t* __restrict__ pos_up, const double* __restrict__ val,
                       double* __restrict__ g64, int* errflag) {
  __shared__ double Ash[kFsaiWarps][kFsaiMax][kFsaiMax + 1];
  __shared__ int32_t Psh[kFsaiWarps][kFsaiMax];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double (*A)[kFsaiMax + 1] = Ash[wid];
  int32_t* P = Psh[wid];
  const int64_t warps = (int64_t)gridDim.x * kFsaiWarps;
  const int64_t nrows = *count;
  for (int64_t li = blockIdx.x * (int64_t)kFsaiWarps + wid; li < nrows; li += warps) {
    const int64_t i = rows[li];
    const int32_t k0 = rowptr[i], kd = dpos[i];
    const int k = kd - k0 + 1;
    if (k > kFsaiMax) {
      if (lane == 0) atomicOr(errflag, 8);
      continue;
    }
    __syncwarp();
    if (lane < k) P[lane] = col[k0 + lane];
    __syncwarp();
    fsai_gather(lane, k, P, rowptr, col, val, A, 0.0);
    __syncwarp();
    double dmax = lane < k ? A[lane][lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if (!fsai_cholesky(lane, k, A, kPivotRel * dmax)) {
      __syncwarp();
      fsai_gather(lane, k, P, rowptr, col, val, A, kShiftRel * dmax);
      __syncwarp();
      fsai_cholesky(lane, k, A, 0.0);
    }
    // back substitution C^T g = e_k; lane a holds rhs_a, then g_a
    double rhs = (lane == k - 1) ? 1.0 : 0.0;
    double g = 0.0;
    for (int j = k - 1; j >= 0; --j) {
      double gj = 0.0;
      if (lane == j) gj = rhs / A[j][j];
      gj = __shfl_sync(0xffffffffu, gj, j);
      if (lane == j) g = gj;
      if (lane < j) rhs -= A[j][lane] * gj;
    }
    if (lane < k) {
      const int32_t pos = k0 + lane;
      g64[pos] = g;
      if (lane < k - 1) {  // transpose slot: entry (P[lane], i) in row P[lane]
        const int32_t tp = pos_up[eid[pos]];
        g64[tp] = g;
      }
    }
  }
}

// Thread-per-row FSAI setup for rows with k <= kFsaiThread: every FP64
// instruction of a warp works on 32 rows (GB300's FP64 pipe is narrow, so
// idle lanes cost as much as busy ones).  Each thread keeps the packed lower
// triangle of its k x k block in shared memory, interleaved across threads
// (element e of thread t at A[e * blockDim + t]) so that accesses do not
// conflict.  Rows with k > kFsaiThread go to a list for the warp-per-row
// kernel above.
// k <= 12 covers ~97% of the rows of the Delaunay meshes here (p99 13, max
// 14); 78 packed doubles per thread let 5 blocks of 64 threads share an SM
// (16 allowed only 3: the kernel waits on shared memory and FP64 latency)
#ifndef DEC_FSAI_THREAD_K
#define DEC_FSAI_THREAD_K 12
#endif
constexpr int kFsaiThread = DEC_FSAI_THREAD_K;
constexpr int kFsaiTpb = 64;
constexpr int kPacked = kFsaiThread * (kFsaiThread + 1) / 2;

__device__ __forceinline__ int tri(int a, int b) { return a * (a + 1) / 2 + b; }

template <typename T>
__device__ void fsai_gather_thread(int k, const int32_t* P, int stride,
                                   const int32_t* __restrict__ rowptr,
                                   const int32_t* __restrict__ dpos,
                                   const int32_t* __restrict__ col,
                                   const double* __restrict__ val, T* A, T shift) {
  for (int a = 0; a < k; ++a) {
    for (int b = 0; b <= a; ++b) A[tri(a, b) * stride] = T(0);
    const int32_t r = P[a * stride];
    // lower part of row r (columns <= r, sorted) merged with P[0..a]
    int b = 0;
    const int32_t kend = dpos[r];
    for (int32_t kk = rowptr[r]; kk <= kend; ++kk) {
      const int32_t c = col[kk];
      while (b < a && P[b * stride] < c) ++b;
      if (P[b * stride] == c) A[tri(a, b) * stride] = (T)val[kk];
    }
    A[tri(a, a) * stride] += shift;
  }
}

template <typename T>
__device__ bool fsai_chol_thread(int k, T* A, int stride, T pivot_min) {
  for (int c = 0; c < k; ++c) {
    const T d = A[tri(c, c) * stride];
    if (!(d > pivot_min)) return false;
    const T lc = sqrt(d);
    const T inv = T(1) / lc;
    A[tri(c, c) * stride] = lc;
    for (int r = c + 1; r < k; ++r) A[tri(r, c) * stride] *= inv;
    for (int r = c + 1; r < k; ++r) {
      const T lrc = A[tri(r, c) * stride];
      for (int q = c + 1; q <= r; ++q) A[tri(r, q) * stride] -= lrc * A[tri(q, c) * stride];
    }
  }
  return true;
}

// T = double: the factor of the FP64 solves.  T = float: the factor the
// batched solve keeps only in BF16 (its rounding dominates the FP32 one),
// with the pivot guard of the per-instance FP32 factors (pivot <= 1e-6
// max(diag): factored again with a 1e-5 max(diag) shift).
template <typename T>
__global__ void __launch_bounds__(kFsaiTpb)
fsai_setup_thread_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                         const int32_t* __restrict__ col, const int32_t* __restrict__ eid,
                         const int32_t* __restrict__ dpos,
                         const int32_t* __restrict__ pos_up,
                         const double* __restrict__ val, double* __restrict__ g64,
                         int32_t* __restrict__ big_rows, int32_t* __restrict__ big_count) {
  extern __shared__ double smem[];
  T* A = reinterpret_cast<T*>(smem) + threadIdx.x;         // stride kFsaiTpb
  int32_t* P = (int32_t*)(reinterpret_cast<T*>(smem) + kPacked * kFsaiTpb) + threadIdx.x;
  constexpr bool f64 = sizeof(T) == sizeof(double);
  const T pivot_rel = f64 ? T(kPivotRel) : T(1e-6), shift_rel = f64 ? T(kShiftRel) : T(1e-5);
  const int stride = kFsaiTpb;
  for (int64_t i = blockIdx.x * (int64_t)kFsaiTpb + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kFsaiTpb) {
    const int32_t k0 = rowptr[i], kd = dpos[i];
    const int k = kd - k0 + 1;
    if (k > kFsaiThread) {
      big_rows[atomicAdd(big_count, 1)] = (int32_t)i;
      continue;
    }
    for (int a = 0; a < k; ++a) P[a * stride] = col[k0 + a];
    fsai_gather_thread<T>(k, P, stride, rowptr, dpos, col, val, A, T(0));
    T dmax = T(0);
    for (int a = 0; a < k; ++a) dmax = fmax(dmax, A[tri(a, a) * stride]);
    if (!fsai_chol_thread<T>(k, A, stride, pivot_rel * dmax)) {
      fsai_gather_thread<T>(k, P, stride, rowptr, dpos, col, val, A, shift_rel * dmax);
      fsai_chol_thread<T>(k, A, stride, T(0));
    }
    // C^T g = e_k, g_j stored over the used diagonal slot C_jj
    for (int j = k - 1; j >= 0; --j) {
      T sum = (j == k - 1) ? T(1) : T(0);
      for (int r = j + 1; r < k; ++r) sum -= A[tri(r, j) * stride] * A[tri(r, r) * stride];
      A[tri(j, j) * stride] = sum / A[tri(j, j) * stride];
    }
    for (int a = 0; a < k; ++a) {
      const double g = (double)A[tri(a, a) * stride];
      g64[k0 + a] = g;
      if (a < k - 1) g64[pos_up[eid[k0 + a]]] = g;
    }
  }
}

static unsigned grid_rows(const dec_ctx* ctx, int64_t work, int per_block) {
  int64_t g = (work + per_block - 1) / per_block;
  int64_t cap = (int64_t)ctx->num_sms * 32;
  return (unsigned)std::max<int64_t>(1, std::min(g, cap));
}

dec_status build_values(dec_ctx* ctx, int inst) {
  const int64_t n = ctx->n, nnz = ctx->nnz;
  const int vs = value_set(ctx, inst);               // value set
  const int ts = ctx->n_sets > 1 ? inst : 0;        // Dirichlet set
  const int fs = ctx->n_fields > 1 ? inst : 0;      // conductivity field
  double* val = ctx->val64.p + (int64_t)vs * nnz;
  laplacian_values_kernel<<<grid_rows(ctx, n, 256), 256, 0, ctx->stream>>>(
      n, ctx->rowptr.p, ctx->col.p, ctx->eid.p, ctx->dpos.p, ctx->tag.p,
      ctx->w.p + (int64_t)fs * ctx->ne, ctx->first_cut.p, ctx->n_scales > 1 ? inst : 0,
      ctx->T0.p + (int64_t)ts * n, val, ctx->b.p + (int64_t)inst * n);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 1;
  if (inst == vs) {   // first instance of this value set: solver copies
    const int64_t tot = ctx->sellL.total;
    DEC_TRY_STATUS(scatter_values<double>(ctx, ctx->sellL, val, ctx->sL64.p + (int64_t)vs * tot));
    DEC_TRY_STATUS(scatter_values<float>(ctx, ctx->sellL, val, ctx->sL32.p + (int64_t)vs * tot));
  }
  return DEC_OK;
}

// Value set 0 = the uncracked operator (no edge cut in any state) with the
// first Dirichlet set: the matrix whose FSAI factor a batched solve shares.
dec_status build_values_uncracked(dec_ctx* ctx) {
  const int64_t n = ctx->n;
  laplacian_values_kernel<<<grid_rows(ctx, n, 256), 256, 0, ctx->stream>>>(
      n, ctx->rowptr.p, ctx->col.p, ctx->eid.p, ctx->dpos.p, ctx->tag.p, ctx->w.p,
      ctx->first_cut.p, -1, ctx->T0.p, ctx->val64.p, ctx->b.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 1;
  const int64_t tot = ctx->sellL.total;
  DEC_TRY_STATUS(scatter_values<double>(ctx, ctx->sellL, ctx->val64.p, ctx->sL64.p));
  DEC_TRY_STATUS(scatter_values<float>(ctx, ctx->sellL, ctx->val64.p, ctx->sL32.p));
  (void)tot;
  return DEC_OK;
}

dec_status build_precond(dec_ctx* ctx, int vs) {
  const int64_t n = ctx->n, nnz = ctx->nnz;
  const double* val = ctx->val64.p + (int64_t)vs * nnz;
  cudaStream_t s = ctx->stream;
  if (ctx->precond == DEC_PRECOND_JACOBI) {
    jacobi_kernel<<<grid_rows(ctx, n, 256), 256, 0, s>>>(
        n, ctx->dpos.p, val, ctx->dinv64.p + (int64_t)vs * n, ctx->dinv32.p + (int64_t)vs * n);
    DEC_TRY(cudaGetLastError());
    ctx->launches += 1;
    return DEC_OK;
  }
  double* g = ctx->g64.p + (int64_t)vs * nnz;
  DEC_TRY(ctx->big_rows.ensure(n + 1));
  int32_t* big_count = ctx->big_rows.p + n;
  DEC_TRY(cudaMemsetAsync(ctx->errflag.p, 0, sizeof(int), s));
  DEC_TRY(cudaMemsetAsync(big_count, 0, sizeof(int32_t), s));
  // the batched solve keeps only a BF16 copy of its shared factor: FP32 set-up
  const bool f32 = ctx->precond == DEC_PRECOND_FSAI_SHARED;
  const size_t smem = (size_t)kPacked * kFsaiTpb * (f32 ? sizeof(float) : sizeof(double)) +
                      (size_t)kFsaiThread * kFsaiTpb * sizeof(int32_t);
  const void* fk = f32 ? (const void*)fsai_setup_thread_kernel<float>
                       : (const void*)fsai_setup_thread_kernel<double>;
  DEC_TRY(cudaFuncSetAttribute(fk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned gt = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((n + kFsaiTpb - 1) / kFsaiTpb,
                           (int64_t)ctx->num_sms * std::max<int64_t>(1, (220 << 10) / smem)));
  if (f32)
    fsai_setup_thread_kernel<float><<<gt, kFsaiTpb, smem, s>>>(
        n, ctx->rowptr.p, ctx->col.p, ctx->eid.p, ctx->dpos.p, ctx->pos_up.p, val, g,
        ctx->big_rows.p, big_count);
  else
    fsai_setup_thread_kernel<double><<<gt, kFsaiTpb, smem, s>>>(
        n, ctx->rowptr.p, ctx->col.p, ctx->eid.p, ctx->dpos.p, ctx->pos_up.p, val, g,
        ctx->big_rows.p, big_count);
  fsai_setup_list_kernel<<<(unsigned)ctx->num_sms * 4, 32 * kFsaiWarps, 0, s>>>(
      ctx->big_rows.p, big_count, ctx->rowptr.p, ctx->col.p, ctx->eid.p, ctx->dpos.p,
      ctx->pos_up.p, val, g, ctx->errflag.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 2;
  const int64_t tlo = ctx->sellLo.total, tup = ctx->sellUp.total;
  DEC_TRY_STATUS(scatter_values<double>(ctx, ctx->sellLo, g, ctx->sGlo64.p + (int64_t)vs * tlo));
  DEC_TRY_STATUS(scatter_values<double>(ctx, ctx->sellUp, g, ctx->sGup64.p + (int64_t)vs * tup));
  DEC_TRY_STATUS(scatter_values<__nv_bfloat16>(ctx, ctx->sellLo, g, ctx->sGlo16.p + (int64_t)vs * tlo));
  DEC_TRY_STATUS(scatter_values<__nv_bfloat16>(ctx, ctx->sellUp, g, ctx->sGup16.p + (int64_t)vs * tup));
  int flag = 0;
  DEC_TRY(cudaMemcpyAsync(&flag, ctx->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaStreamSynchronize(s));
  if (flag & 8)
    return ctx->fail(DEC_ERR_LIMIT, "an FSAI row has more than 32 lower-pattern entries");
  return DEC_OK;
}

// ------------------------------------------------------ crack update
// A crack sets the *1 of one edge e = (i, j) to 0 (Sec. 2.3, 2.5): only rows
// and columns i and j of L change (L_ii, L_jj, L_ij, L_ji, plus b_i, b_j
// through Dirichlet neighbours).  Threads 0 and 1 recompute rows i and j
// exactly as a full build does, with their solver copies and Jacobi entries;
// thread 0 then lists the FSAI rows whose principal block L[P_r, P_r] holds
// i or j (P_r = lower pattern of row r): r = i, j and their neighbours of
// larger id.
__global__ void crack_rows_kernel(int64_t e, const int32_t* __restrict__ E,
                                  const int32_t* __restrict__ rowptr,
                                  const int32_t* __restrict__ col,
                                  const int32_t* __restrict__ eid,
                                  const int32_t* __restrict__ dpos,
                                  const uint8_t* __restrict__ tag, const double* __restrict__ w,
                                  const uint8_t* __restrict__ fc, const double* __restrict__ T0,
                                  double* __restrict__ val, double* __restrict__ b,
                                  const int32_t* __restrict__ sell_pos, double* __restrict__ sL64,
                                  float* __restrict__ sL32, double* __restrict__ dinv64,
                                  float* __restrict__ dinv32, int32_t* __restrict__ list,
                                  int32_t* __restrict__ count) {
  if (threadIdx.x < 2) {
    const int64_t i = E[2 * e + threadIdx.x];
    laplacian_row(i, rowptr, col, eid, dpos, tag, w, fc, 0, T0, val, b);
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int32_t p = sell_pos[k];
      if (p >= 0) {
        sL64[p] = val[k];
        sL32[p] = (float)val[k];
      }
    }
    if (dinv64) {
      const double d = 1.0 / val[dpos[i]];
      dinv64[i] = d;
      dinv32[i] = (float)d;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t c = 0;
    for (int h = 0; h < 2; ++h) {
      const int32_t i = E[2 * e + h];
      list[c++] = i;
      for (int32_t k = dpos[i] + 1; k < rowptr[i + 1]; ++k) list[c++] = col[k];
    }
    *count = c;
  }
}

// solver copies (FP64 and BF16, both halves) of the listed FSAI rows
__global__ void fsai_rows_scatter_kernel(const int32_t* __restrict__ list,
                                         const int32_t* __restrict__ count,
                                         const int32_t* __restrict__ rowptr,
                                         const int32_t* __restrict__ dpos,
                                         const int32_t* __restrict__ eid,
                                         const int32_t* __restrict__ pos_up,
                                         const double* __restrict__ g64,
                                         const int32_t* __restrict__ lo_pos,
                                         const int32_t* __restrict__ up_pos,
                                         double* __restrict__ glo64, double* __restrict__ gup64,
                                         __nv_bfloat16* __restrict__ glo16,
                                         __nv_bfloat16* __restrict__ gup16) {
  const int32_t nrows = *count;
  for (int32_t li = threadIdx.x; li < nrows; li += blockDim.x) {
    const int32_t r = list[li];
    for (int32_t k = rowptr[r]; k <= dpos[r]; ++k) {
      const double g = g64[k];
      const int32_t pl = lo_pos[k];
      if (pl >= 0) {
        glo64[pl] = g;
        glo16[pl] = __float2bfloat16_rn((float)g);
      }
      const int32_t tp = k == dpos[r] ? k : pos_up[eid[k]];
      const int32_t pu = up_pos[tp];
      if (pu >= 0) {
        gup64[pu] = g64[tp];
        gup16[pu] = __float2bfloat16_rn((float)g64[tp]);
      }
    }
  }
}

dec_status crack_update(dec_ctx* ctx, int64_t e) {
  cudaStream_t s = ctx->stream;
  const bool jac = ctx->precond == DEC_PRECOND_JACOBI;
  // the list holds at most 2 + deg(i) + deg(j) <= nnz rows
  DEC_TRY(ctx->big_rows.ensure(ctx->nnz + 1));
  int32_t* list = ctx->big_rows.p;
  int32_t* count = ctx->big_rows.p + ctx->nnz;
  crack_rows_kernel<<<1, 32, 0, s>>>(
      e, ctx->E.p, ctx->rowptr.p, ctx->col.p, ctx->eid.p, ctx->dpos.p, ctx->tag.p, ctx->w.p,
      ctx->first_cut.p, ctx->T0.p, ctx->val64.p, ctx->b.p, ctx->sellL.pos.p, ctx->sL64.p,
      ctx->sL32.p, jac ? ctx->dinv64.p : nullptr, jac ? ctx->dinv32.p : nullptr, list, count);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 1;
  if (jac) return DEC_OK;
  DEC_TRY(cudaMemsetAsync(ctx->errflag.p, 0, sizeof(int), s));
  fsai_setup_list_kernel<<<16, 32 * kFsaiWarps, 0, s>>>(
      list, count, ctx->rowptr.p, ctx->col.p, ctx->eid.p, ctx->dpos.p, ctx->pos_up.p,
      ctx->val64.p, ctx->g64.p, ctx->errflag.p);
  fsai_rows_scatter_kernel<<<1, 64, 0, s>>>(
      list, count, ctx->rowptr.p, ctx->dpos.p, ctx->eid.p, ctx->pos_up.p, ctx->g64.p,
      ctx->sellLo.pos.p, ctx->sellUp.pos.p, ctx->sGlo64.p, ctx->sGup64.p, ctx->sGlo16.p,
      ctx->sGup16.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 2;
  return DEC_OK;
}

}  // namespace dec
