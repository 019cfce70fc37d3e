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
// diagonal on: G^T).  The batched solve uses the same builder with slices of
// C = 32 / (threads per row) rows and windows of R rows taken in a spatial
// (Morton) order of the nodes instead of the natural one.  Each gets its own permutation, slice pointers and
// column array; `pos` maps a CSR slot to its SELL slot (-1 if not present),
// so value arrays built in CSR order are scattered once per build.
#include "dec_internal.cuh"

#include <algorithm>

namespace dec {

constexpr int kWindow = 512;

// Entries of row i that a layout of `kind` stores, in CSR order:
//   0: the whole row; 1: lower half incl. diagonal (G); 2: upper half incl.
//   diagonal (G^T); 3: off-diagonal entries, none on Dirichlet rows (edge
//   form of the batched solve); 4: off-diagonal entries whose column is not
//   a Dirichlet node, none on Dirichlet rows (CSR form of the batched solve,
//   whose Dirichlet columns carry no value).
__device__ __forceinline__ bool kind_keeps(int kind, int32_t k, int32_t kd, int32_t c,
                                           const uint8_t* tag) {
  if (kind == 0) return true;
  if (kind == 1) return k <= kd;
  if (kind == 2) return k >= kd;
  if (kind == 3) return k != kd;
  return k != kd && tag[c] != DEC_NODE_DIRICHLET;
}

__device__ __forceinline__ int32_t kind_len(int kind, const int32_t* rowptr,
                                            const int32_t* dpos, const int32_t* col,
                                            const uint8_t* tag, int64_t i) {
  const int32_t k0 = rowptr[i], k1 = rowptr[i + 1], kd = dpos[i];
  if (kind == 0) return k1 - k0;
  if (kind == 1) return kd - k0 + 1;
  if (kind == 2) return k1 - kd;
  if (tag[i] == DEC_NODE_DIRICHLET) return 0;
  if (kind == 3) return k1 - k0 - 1;
  int32_t l = 0;
  for (int32_t k = k0; k < k1; ++k) l += kind_keeps(4, k, kd, col[k], tag) ? 1 : 0;
  return l;
}

// Rank the rows of each window of R rows (natural order, or the order
// `order` gives) by (length desc, position asc).  One block per window,
// blockDim = R.
__global__ void sell_sort_kernel(int kind, int64_t n, const int32_t* __restrict__ order,
                                 const int32_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ dpos,
                                 const int32_t* __restrict__ col,
                                 const uint8_t* __restrict__ tag,
                                 int32_t* __restrict__ perm, int32_t* __restrict__ len_out) {
  extern __shared__ int32_t wlen[];
  const int R = blockDim.x;
  const int64_t at = (int64_t)blockIdx.x * R + threadIdx.x;
  int32_t row = -1, l = -1;
  if (at < n) {
    row = order ? order[at] : (int32_t)at;
    l = kind_len(kind, rowptr, dpos, col, tag, row);
  }
  wlen[threadIdx.x] = l;
  __syncthreads();
  int rank = 0;
  for (int j = 0; j < R; ++j) {
    const int32_t lj = wlen[j];
    rank += (lj > l) || (lj == l && j < (int)threadIdx.x);
  }
  const int64_t slot = (int64_t)blockIdx.x * R + rank;
  perm[slot] = row;
  len_out[slot] = l < 0 ? 0 : l;   // length of the row in slot order
}

// entries of slice s = C * (length of its first, longest row)
__global__ void sell_width_kernel(int64_t nslices, int C, const int32_t* __restrict__ len_sorted,
                                  uint32_t* __restrict__ size) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s <= nslices;
       s += (int64_t)gridDim.x * blockDim.x)
    size[s] = s < nslices ? (uint32_t)C * (uint32_t)len_sorted[(int64_t)C * s] : 0u;
}

__global__ void sell_fill_kernel(int kind, int64_t nslices, int C,
                                 const int32_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ dpos,
                                 const int32_t* __restrict__ csr_col,
                                 const uint8_t* __restrict__ tag,
                                 const int32_t* __restrict__ perm,
                                 const int32_t* __restrict__ sptr,
                                 int32_t* __restrict__ scol, int32_t* __restrict__ pos) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t s = t / C;
  const int lane = (int)(t % C);
  if (s >= nslices) return;
  const int32_t r = perm[t];
  const int32_t base = sptr[s];
  const int32_t w = (sptr[s + 1] - base) / C;
  int32_t j = 0;
  if (r >= 0 && !((kind == 3 || kind == 4) && tag[r] == DEC_NODE_DIRICHLET)) {
    const int32_t kd = dpos[r];
    for (int32_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
      if (!kind_keeps(kind, k, kd, csr_col[k], tag)) continue;
      const int32_t p = base + C * j + lane;
      scol[p] = csr_col[k];
      pos[k] = p;
      ++j;
    }
  }
  // padding: value 0, a column already in cache (the row itself)
  for (; j < w; ++j) scol[base + C * j + lane] = r >= 0 ? r : 0;
}

dec_status build_sell(dec_ctx* ctx, int kind, SellLayout& L, int C, int R,
                      const int32_t* order) {
  const int64_t n = ctx->n;
  cudaStream_t s = ctx->stream;
  if (C < 1 || R % C != 0 || R > 1024) return ctx->fail(DEC_ERR_ARG, "build_sell: bad shape");
  const int64_t nwin = (n + R - 1) / R;
  L.C = C;
  L.R = R;
  L.nslices = nwin * (R / C);
  const int64_t slots = nwin * R;
  DEC_TRY(L.perm.ensure(slots));
  DEC_TRY(L.len.ensure(slots));
  DEC_TRY(L.sptr.ensure(L.nslices + 1));
  DEC_TRY(L.pos.ensure(ctx->nnz));
  sell_sort_kernel<<<(unsigned)nwin, R, R * sizeof(int32_t), s>>>(
      kind, n, order, ctx->rowptr.p, ctx->dpos.p, ctx->col.p, ctx->tag.p, L.perm.p, L.len.p);
  sell_width_kernel<<<(unsigned)std::min<int64_t>((L.nslices + 256) / 256, 4096), 256, 0, s>>>(
      L.nslices, C, L.len.p, (uint32_t*)L.sptr.p);
  DEC_TRY(cudaGetLastError());
  DEC_TRY(ctx->scan_tmp.ensure(scan_tmp_size(L.nslices + 1)));
  DEC_TRY(exclusive_scan_u32((const uint32_t*)L.sptr.p, (uint32_t*)L.sptr.p, L.nslices + 1,
                             ctx->scan_tmp.p, ctx->scan_tmp.cap, s));
  uint32_t total = 0;
  DEC_TRY(cudaMemcpyAsync(&total, L.sptr.p + L.nslices, sizeof(uint32_t),
                          cudaMemcpyDeviceToHost, s));
  DEC_TRY(cudaStreamSynchronize(s));
  if (total >= (uint32_t)INT32_MAX)
    return ctx->fail(DEC_ERR_LIMIT, "sliced layout: more than 2^31 - 1 entries");
  L.total = total;
  DEC_TRY(L.col.ensure(total));
  DEC_TRY(cudaMemsetAsync(L.pos.p, 0xff, sizeof(int32_t) * ctx->nnz, s));
  sell_fill_kernel<<<(unsigned)((slots + 255) / 256), 256, 0, s>>>(
      kind, L.nslices, C, ctx->rowptr.p, ctx->dpos.p, ctx->col.p, ctx->tag.p, L.perm.p,
      L.sptr.p, L.col.p, L.pos.p);
  DEC_TRY(cudaGetLastError());
  ctx->launches += 6;  // sort, widths, scan (3), fill
  return DEC_OK;
}

dec_status build_sell_layouts(dec_ctx* ctx) {
  DEC_TRY_STATUS(build_sell(ctx, 0, ctx->sellL, 32, kWindow, nullptr));
  DEC_TRY_STATUS(build_sell(ctx, 1, ctx->sellLo, 32, kWindow, nullptr));
  DEC_TRY_STATUS(build_sell(ctx, 2, ctx->sellUp, 32, kWindow, nullptr));
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
