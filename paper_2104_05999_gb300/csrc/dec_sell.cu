// dec_sell.cu - the solver's storage layout: sliced ELLPACK with slices of
// 32 rows and rows sorted by length inside windows of 512 rows (SELL-32-512).
//
// One warp processes one slice, one lane per row, so every FMA lane does
// useful work (GB300's FP64 pipe is narrow: a half-empty FP64 warp
// instruction costs as much as a full one) and the column / value loads of a
// slice are contiguous (entry j of the slice's 32 rows is stored at
// sptr[s] + 32 j + lane).  Rows are padded to the longest row of their slice;
// sorting inside 512-row windows keeps that padding near 3 % on the
// Delaunay meshes while gathers stay inside a window of the lattice order.
//
// Three matrices share the CSR structure of L: L itself, the lower half of
// the FSAI factor (entries up to the diagonal: G) and the upper half (from the
// diagonal on: G^T).  Each gets its own permutation, slice pointers and
// column array; `pos` maps a CSR slot to its SELL slot (-1 if not present),
// so value arrays built in CSR order are scattered once per build.
#include "dec_internal.cuh"

#include <algorithm>

namespace dec {

constexpr int kWindow = 512;

// kind 0: whole row; 1: lower half incl. diagonal; 2: upper half incl. diagonal
__device__ __forceinline__ void row_range(int kind, const int32_t* rowptr,
                                          const int32_t* dpos, int64_t i,
                                          int32_t* k0, int32_t* k1) {
  if (kind == 0) { *k0 = rowptr[i]; *k1 = rowptr[i + 1]; }
  else if (kind == 1) { *k0 = rowptr[i]; *k1 = dpos[i] + 1; }
  else { *k0 = dpos[i]; *k1 = rowptr[i + 1]; }
}

// rank rows of each 512-row window by (length desc, row asc)
__global__ void __launch_bounds__(kWindow)
sell_sort_kernel(int kind, int64_t n, const int32_t* __restrict__ rowptr,
                 const int32_t* __restrict__ dpos, int32_t* __restrict__ perm,
                 int32_t* __restrict__ len_out) {
  __shared__ int32_t len[kWindow];
  const int64_t row = (int64_t)blockIdx.x * kWindow + threadIdx.x;
  int32_t l = -1;
  if (row < n) {
    int32_t k0, k1;
    row_range(kind, rowptr, dpos, row, &k0, &k1);
    l = k1 - k0;
  }
  len[threadIdx.x] = l;
  __syncthreads();
  int rank = 0;
  for (int j = 0; j < kWindow; ++j) {
    const int32_t lj = len[j];
    rank += (lj > l) || (lj == l && j < (int)threadIdx.x);
  }
  const int64_t slot = (int64_t)blockIdx.x * kWindow + rank;
  perm[slot] = row < n ? (int32_t)row : -1;
  len_out[slot] = l < 0 ? 0 : l;   // length of the row in slot order
}

// entries of slice s = 32 * (length of its first, longest row)
__global__ void sell_width_kernel(int64_t nslices, const int32_t* __restrict__ len_sorted,
                                  uint32_t* __restrict__ size) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s <= nslices;
       s += (int64_t)gridDim.x * blockDim.x)
    size[s] = s < nslices ? 32u * (uint32_t)len_sorted[32 * s] : 0u;
}

__global__ void sell_fill_kernel(int kind, int64_t nslices,
                                 const int32_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ dpos,
                                 const int32_t* __restrict__ csr_col,
                                 const int32_t* __restrict__ perm,
                                 const int32_t* __restrict__ sptr,
                                 int32_t* __restrict__ scol, int32_t* __restrict__ pos) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t s = t >> 5;
  const int lane = (int)(t & 31);
  if (s >= nslices) return;
  const int32_t r = perm[32 * s + lane];
  const int32_t base = sptr[s];
  const int32_t w = (sptr[s + 1] - base) >> 5;
  int32_t k0 = 0, k1 = 0;
  if (r >= 0) row_range(kind, rowptr, dpos, r, &k0, &k1);
  for (int32_t j = 0; j < w; ++j) {
    const int32_t p = base + 32 * j + lane;
    if (r >= 0 && j < k1 - k0) {
      scol[p] = csr_col[k0 + j];
      pos[k0 + j] = p;
    } else {
      scol[p] = r >= 0 ? r : 0;   // padding: value 0, a column already in cache
    }
  }
}

dec_status build_sell(dec_ctx* ctx, int kind, SellLayout& L) {
  const int64_t n = ctx->n;
  cudaStream_t s = ctx->stream;
  const int64_t nwin = (n + kWindow - 1) / kWindow;
  L.nslices = nwin * (kWindow / 32);
  const int64_t slots = L.nslices * 32;
  DEC_TRY(L.perm.ensure(slots));
  DEC_TRY(L.len.ensure(slots));
  DEC_TRY(L.sptr.ensure(L.nslices + 1));
  DEC_TRY(L.pos.ensure(ctx->nnz));
  sell_sort_kernel<<<(unsigned)nwin, kWindow, 0, s>>>(kind, n, ctx->rowptr.p, ctx->dpos.p,
                                                     L.perm.p, L.len.p);
  sell_width_kernel<<<(unsigned)std::min<int64_t>((L.nslices + 256) / 256, 4096), 256, 0, s>>>(
      L.nslices, L.len.p, (uint32_t*)L.sptr.p);
  DEC_TRY(cudaGetLastError());
  DEC_TRY(ctx->scan_tmp.ensure(scan_tmp_size(L.nslices + 1)));
  DEC_TRY(exclusive_scan_u32((const uint32_t*)L.sptr.p, (uint32_t*)L.sptr.p, L.nslices + 1,
                             ctx->scan_tmp.p, ctx->scan_tmp.cap, s));
  int32_t total = 0;
  DEC_TRY(cudaMemcpyAsync(&total, L.sptr.p + L.nslices, sizeof(int32_t),
                          cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaStreamSynchronize(s));
  L.total = total;
  DEC_TRY(L.col.ensure(total));
  DEC_TRY(cudaMemsetAsync(L.pos.p, 0xff, sizeof(int32_t) * ctx->nnz, s));
  sell_fill_kernel<<<(unsigned)((slots + 255) / 256), 256, 0, s>>>(
      kind, L.nslices, ctx->rowptr.p, ctx->dpos.p, ctx->col.p, L.perm.p, L.sptr.p,
      L.col.p, L.pos.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 6;  // sort, widths, scan (3), fill
  return DEC_OK;
}

dec_status build_sell_layouts(dec_ctx* ctx) {
  DEC_TRY_STATUS(build_sell(ctx, 0, ctx->sellL));
  DEC_TRY_STATUS(build_sell(ctx, 1, ctx->sellLo));
  DEC_TRY_STATUS(build_sell(ctx, 2, ctx->sellUp));
  return DEC_OK;
}

// scatter CSR-ordered values into a SELL value array (padding stays 0)
template <typename S, typename T>
__global__ void sell_scatter_kernel(int64_t nnz, const int32_t* __restrict__ pos,
                                    const S* __restrict__ v, T* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = pos[k];
    if (p >= 0) out[p] = (T)v[k];
  }
}

template <>
__global__ void sell_scatter_kernel<double, __nv_bfloat16>(int64_t nnz,
                                                           const int32_t* __restrict__ pos,
                                                           const double* __restrict__ v,
                                                           __nv_bfloat16* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = pos[k];
    if (p >= 0) out[p] = __float2bfloat16_rn((float)v[k]);
  }
}

template <typename T>
dec_status scatter_values(dec_ctx* ctx, const SellLayout& L, const double* csr_val, T* out) {
  cudaStream_t s = ctx->stream;
  DEC_TRY(cudaMemsetAsync(out, 0, sizeof(T) * L.total, s));
  const int64_t nnz = ctx->nnz;
  unsigned g = (unsigned)std::min<int64_t>((nnz + 255) / 256, (int64_t)ctx->num_sms * 16);
  sell_scatter_kernel<double, T><<<g, 256, 0, s>>>(nnz, L.pos.p, csr_val, out);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 1;
  return DEC_OK;
}

template dec_status scatter_values<double>(dec_ctx*, const SellLayout&, const double*, double*);
template dec_status scatter_values<float>(dec_ctx*, const SellLayout&, const double*, float*);
template dec_status scatter_values<__nv_bfloat16>(dec_ctx*, const SellLayout&, const double*,
                                                  __nv_bfloat16*);

}  // namespace dec
